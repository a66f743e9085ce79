"""Hyper-dual numbers and a value-only strain energy, used to pin the oracle's derivatives.

Hyper-dual numbers (Fike & Alonso, AIAA 2011-886) a + b e1 + c e2 + d e1e2 with
e1^2 = e2^2 = 0 carry exact first and mixed second derivatives through any smooth
computation, with no step-size error. Seeding F_a with e1 and F_b with e2 and evaluating
Psi(F) returns dPsi/dF_a in the e1 part and d2Psi/dF_a dF_b in the e1e2 part.

``psi_hd`` evaluates the strain energy from its definitions only: C = F^T F, the
invariants of eq. 454, the isochoric invariants I_m I3^alpha_m of App. A.2 (computed
through I3 = det C, not J), the MICNN forward pass of eq. icnn and the volumetric
penalty. It contains no derivative formula, so it is independent of the oracle's
hand-derived kinematics and of Algorithm 4.

Components are numpy arrays, so one call evaluates a batch of seedings at once.
"""
from __future__ import annotations

import numpy as np


class HD:
    __slots__ = ("r", "e1", "e2", "e12")

    def __init__(self, r, e1=0.0, e2=0.0, e12=0.0):
        self.r, self.e1, self.e2, self.e12 = r, e1, e2, e12

    @staticmethod
    def lift(x):
        return x if isinstance(x, HD) else HD(x)

    def __add__(self, o):
        o = HD.lift(o)
        return HD(self.r + o.r, self.e1 + o.e1, self.e2 + o.e2, self.e12 + o.e12)

    __radd__ = __add__

    def __neg__(self):
        return HD(-self.r, -self.e1, -self.e2, -self.e12)

    def __sub__(self, o):
        return self + (-HD.lift(o))

    def __rsub__(self, o):
        return HD.lift(o) + (-self)

    def __mul__(self, o):
        o = HD.lift(o)
        return HD(self.r * o.r, self.r * o.e1 + self.e1 * o.r, self.r * o.e2 + self.e2 * o.r,
                  self.r * o.e12 + self.e1 * o.e2 + self.e2 * o.e1 + self.e12 * o.r)

    __rmul__ = __mul__

    def apply(self, f, f1, f2):
        """g(x) for g with value f, first derivative f1 and second derivative f2 at x.r."""
        return HD(f, f1 * self.e1, f1 * self.e2, f1 * self.e12 + f2 * self.e1 * self.e2)

    def recip(self):
        r = self.r
        return self.apply(1.0 / r, -1.0 / r ** 2, 2.0 / r ** 3)

    def __truediv__(self, o):
        return self * HD.lift(o).recip()

    def __rtruediv__(self, o):
        return HD.lift(o) * self.recip()

    def __pow__(self, p: float):
        r = self.r
        return self.apply(r ** p, p * r ** (p - 1), p * (p - 1) * r ** (p - 2))

    def __getitem__(self, idx):
        g = lambda x: x[idx] if np.ndim(x) else x
        return HD(g(self.r), g(self.e1), g(self.e2), g(self.e12))


def hd_exp(x: HD) -> HD:
    e = np.exp(x.r)
    return x.apply(e, e, e)


def hd_log(x: HD) -> HD:
    return x.apply(np.log(x.r), 1.0 / x.r, -1.0 / x.r ** 2)


def hd_softplus(x: HD) -> HD:
    r = x.r
    f = np.maximum(r, 0.0) + np.log1p(np.exp(-np.abs(r)))
    s = 0.5 * (1.0 + np.tanh(0.5 * r))  # logistic
    return x.apply(f, s, s * (1.0 - s))


def hd_matvec(M: np.ndarray, v: HD) -> HD:
    """Real matrix times hyper-dual vector (v components shaped [n, ...])."""
    t = lambda x: np.tensordot(M, x, axes=([1], [0])) if np.ndim(x) else x * M.sum(axis=1)
    return HD(t(v.r), t(v.e1), t(v.e2), t(v.e12))


def hd_stack(items):
    def comp(name):
        vals = [getattr(it, name) for it in items]
        shape = np.broadcast(*[np.asarray(v) for v in vals]).shape
        return np.stack([np.broadcast_to(np.asarray(v, dtype=float), shape) for v in vals])
    return HD(comp("r"), comp("e1"), comp("e2"), comp("e12"))


# ------------------------------------------------------------------- strain energy

def _det3(M):
    """Determinant of a 3x3 nested list of HD entries (rule of Sarrus)."""
    return (M[0][0] * M[1][1] * M[2][2] + M[0][1] * M[1][2] * M[2][0] + M[0][2] * M[1][0] * M[2][1]
            - M[0][2] * M[1][1] * M[2][0] - M[0][0] * M[1][2] * M[2][1] - M[0][1] * M[1][0] * M[2][2])


def kinematic_scalars(F9, kin: int, fibres) -> list:
    """K(F) from definitions (eq. 454; App. A.2), F9 = 9 HD entries, row-major F_iJ."""
    F = [[F9[3 * i + J] for J in range(3)] for i in range(3)]
    C = [[sum((F[k][I] * F[k][J] for k in range(3)), HD(0.0)) for J in range(3)] for I in range(3)]
    I1 = C[0][0] + C[1][1] + C[2][2]
    trC2 = sum((C[I][J] * C[J][I] for I in range(3) for J in range(3)), HD(0.0))
    I2 = 0.5 * (I1 * I1 - trC2)
    I3 = _det3(C)
    J = _det3(F)
    Ib1 = I1 * I3 ** (-1.0 / 3.0)
    Ib2 = I2 * I3 ** (-2.0 / 3.0)
    if kin == 0:
        return [Ib1 - 3.0, Ib2 - 3.0, J - 1.0], J
    if kin == 2:
        return [Ib1 - 3.0, Ib2 ** 1.5 - 3.0 ** 1.5, (J - 1.0) * (J - 1.0)], J
    K = [Ib1, Ib2, J]
    I4s, I5s = [], []
    for A0 in fibres:
        CA = [sum((C[I][M] * float(A0[M]) for M in range(3)), HD(0.0)) for I in range(3)]
        I4s.append(sum((CA[I] * float(A0[I]) for I in range(3)), HD(0.0)))
        I5s.append(sum((CA[I] * CA[I] for I in range(3)), HD(0.0)))
    return K + I4s + I5s, J


def micnn_forward(spec, K: HD) -> HD:
    """eq. icnn forward pass on a stacked HD input K (components shaped [d, ...])."""
    z = hd_softplus(hd_matvec(spec.W1, K) + spec.c[0].reshape((-1,) + (1,) * (np.ndim(K.r) - 1)))
    for k in range(spec.L - 1):
        cb = spec.c[k + 1].reshape((-1,) + (1,) * (np.ndim(K.r) - 1))
        z = hd_softplus(hd_matvec(spec.Ak[k], z) + hd_matvec(spec.Bk[k], K) + cb)
    out = hd_matvec(spec.a[None, :], z) + hd_matvec(spec.b[None, :], K)
    return out[0]


def _sign(x):
    return np.sign(x)


def cann_forward(spec, K: list) -> HD:
    """eq. cann-def from the menus of eq. cann-fs, value only, on a list of HD inputs."""
    out = HD(0.0)
    for m in range(spec.d):
        for k in range(spec.n):
            f0k, p, f2k = (int(v) for v in spec.kinds[k])
            w1, w2 = float(spec.w[m, k, 0]), float(spec.w[m, k, 1])
            x = K[m]
            if f0k == 1:    # Macaulay bracket
                x = x.apply(np.maximum(x.r, 0.0), 0.5 * (1.0 + _sign(x.r)), 0.0)
            elif f0k == 2:  # absolute value
                x = x.apply(np.abs(x.r), _sign(x.r), 0.0)
            y = x
            for _ in range(p - 1):
                y = y * x
            if f2k == 1:
                f = hd_exp(w1 * y) - 1.0
            elif f2k == 2:
                f = -1.0 * hd_log(1.0 - w1 * y)
            else:
                f = w1 * y
            out = out + w2 * f
    return out


def _bspline_hd(k, t, x: HD):
    """Value-only B-spline basis of degree k on knots t at a hyper-dual x (recursion of App. B);
    the indicators are evaluated at the real part (piecewise polynomial)."""
    nk = len(t)
    b = [HD(np.where((t[l] <= x.r) & (x.r < t[l + 1]), 1.0, 0.0)) for l in range(nk - 1)]
    for q in range(1, k + 1):
        b = [(x - t[l]) * (1.0 / (t[l + q] - t[l])) * b[l] + (t[l + q + 1] - x) * (1.0 / (t[l + q + 1] - t[l + 1])) * b[l + 1]
             for l in range(nk - q - 1)]
    return b


def ickan_forward(spec, K: list) -> HD:
    """The KAN of App. B, value only: z_i = sum_j w_s sum_l c_l B_l,k(z_j)."""
    R, k, G = len(spec.widths) - 1, spec.degree, spec.G
    nb = G + k
    z = list(K)
    off = 0
    for r in range(R):
        h = (spec.hi[r] - spec.lo[r]) / G
        t = [spec.lo[r] + (m - k) * h for m in range(G + 2 * k + 1)]
        zn = []
        for i in range(spec.widths[r + 1]):
            acc = HD(0.0)
            for j in range(spec.widths[r]):
                ws, c = spec.params[off], spec.params[off + 1: off + 1 + nb]
                off += 1 + nb
                B = _bspline_hd(k, t, z[j])
                psi = HD(0.0)
                for l in range(nb):
                    psi = psi + float(c[l]) * B[l]
                acc = acc + float(ws) * psi
            zn.append(acc)
        z = zn
    return z[0]


def psi_hd(spec, F9: list, inner=None) -> HD:
    """Psi(F) = N(K(F)) + kappa (J - 1)^2 (stress-free shift not included).
    inner(K_list) -> HD replaces the MICNN when given; CANN specs use eq. cann-def."""
    K, J = kinematic_scalars(F9, spec.kin if inner is None else 1, spec.fibres)
    if inner is not None:
        N = inner(K)
    elif getattr(spec, "inner_name", "micnn") == "cann":
        N = cann_forward(spec, K)
    elif getattr(spec, "inner_name", "micnn") == "ickan":
        N = ickan_forward(spec, K)
    else:
        N = micnn_forward(spec, hd_stack(K))
    return N + spec.kappa * (J - 1.0) * (J - 1.0)


def exact_P_A(spec, F: np.ndarray, inner=None):
    """Exact P[9] and A[81] of psi_hd at one F by hyper-dual seeding (all 81 pairs at once)."""
    F = np.asarray(F, dtype=float).reshape(9)
    a_idx, b_idx = np.meshgrid(np.arange(9), np.arange(9), indexing="ij")
    a_idx, b_idx = a_idx.ravel(), b_idx.ravel()
    F9 = [HD(np.full(81, F[c]), (a_idx == c).astype(float), (b_idx == c).astype(float), 0.0)
          for c in range(9)]
    psi = psi_hd(spec, F9, inner)
    P = psi.e1.reshape(9, 9)[:, 0]
    A = psi.e12.reshape(81)
    return float(psi.r[0]), P, A


def exact_inner(spec, K: np.ndarray):
    """Exact N, dN[d], d2N[d][d] of the eq. icnn forward pass at K by hyper-dual seeding."""
    d = K.size
    a_idx, b_idx = np.meshgrid(np.arange(d), np.arange(d), indexing="ij")
    a_idx, b_idx = a_idx.ravel(), b_idx.ravel()
    Kh = HD(np.repeat(K[:, None], d * d, axis=1), (a_idx[None, :] == np.arange(d)[:, None]).astype(float),
            (b_idx[None, :] == np.arange(d)[:, None]).astype(float), np.zeros((d, d * d)))
    N = micnn_forward(spec, Kh)
    return float(N.r[0]), N.e1.reshape(d, d)[:, 0], N.e12.reshape(d, d)
