"""Seeded synthetic inputs shared by the oracle tests, the CUDA tests and the benchmark.

This module is the one thing both sides use. It holds input recipes only: random
weights, meshes, displacement and deformation fields. It holds none of the method's
arithmetic (no invariants, network evaluation, shape functions or assembly). The one
computation on inputs is a determinant rejection test (``numpy.linalg.det``) that
keeps the drawn deformation gradients orientation-preserving, as the workloads require.

The workloads stand in for the paper's twisted cube and heart meshes with trained
MICNNs (Sec. 4-5): structured unit-cube hex8 meshes and the paper's MICNN family
(Appendix B, eq. icnn; sizes as in the hyper-parameter table and Appendix E), with
random non-negative weights. No dataset is involved.

Draw order for every workload, on one ``numpy.random.Generator(PCG64(seed))``:
weights layer by layer (W1, c1, then A_k, B_k, c_k for k = 2..L, then a, b), then the
displacement or deformation field, then any per-point scalars.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Kinematic layers (input menus) of the strain energy.
KIN_ISO_SHIFTED = 0  # K = (Ibar1 - 3, Ibar2 - 3, J - 1)
KIN_RAW = 1          # K = (Ibar1, Ibar2, J, I4_11..I4_nn, I5_11..I5_nn)
KIN_POLYCONVEX = 2   # K = (Ibar1 - 3, Ibar2^{3/2} - 3^{3/2}, (J - 1)^2), the paper's NCM inputs (App. C)

# Reference structural vectors at +-30 degrees from +x in the x-y plane.
FIBRES_PM30 = np.array([[math.cos(math.pi / 6), math.sin(math.pi / 6), 0.0],
                        [math.cos(math.pi / 6), -math.sin(math.pi / 6), 0.0]])


@dataclass
class ModelSpec:
    """Weights and hyper-parameters of one MICNN strain energy (float64, row-major).

    W1: [W][d]; Ak: [L-1][W][W]; Bk: [L-1][W][d]; c: [L][W]; a: [W]; b: [d].
    """
    d: int
    W: int
    L: int
    kin: int
    fibres: np.ndarray
    W1: np.ndarray
    Ak: np.ndarray
    Bk: np.ndarray
    c: np.ndarray
    a: np.ndarray
    b: np.ndarray
    kappa: float = 0.0
    stress_free: bool = False
    extra: dict = field(default_factory=dict)

    @property
    def n_fib(self) -> int:
        return int(self.fibres.shape[0])

    def theta(self) -> np.ndarray:
        """Flat parameter vector: W1, c1, then per k = 2..L: A_k, B_k, c_k, then a, b."""
        parts = [self.W1.ravel(), self.c[0].ravel()]
        for k in range(self.L - 1):
            parts += [self.Ak[k].ravel(), self.Bk[k].ravel(), self.c[k + 1].ravel()]
        parts += [self.a.ravel(), self.b.ravel()]
        return np.concatenate(parts).astype(np.float64)

    def with_theta(self, theta: np.ndarray) -> "ModelSpec":
        """Copy of this model with the flat parameter vector replaced."""
        d, W, L = self.d, self.W, self.L
        t = np.asarray(theta, dtype=np.float64)
        o = 0

        def take(n, shape):
            nonlocal o
            v = t[o:o + n].reshape(shape).copy()
            o += n
            return v
        W1 = take(W * d, (W, d))
        c = np.zeros((L, W))
        c[0] = take(W, (W,))
        Ak = np.zeros((max(L - 1, 0), W, W))
        Bk = np.zeros((max(L - 1, 0), W, d))
        for k in range(L - 1):
            Ak[k] = take(W * W, (W, W))
            Bk[k] = take(W * d, (W, d))
            c[k + 1] = take(W, (W,))
        a = take(W, (W,))
        b = take(d, (d,))
        assert o == t.size
        return ModelSpec(d, W, L, self.kin, self.fibres.copy(), W1, Ak, Bk, c, a, b, self.kappa,
                         self.stress_free, dict(self.extra))


def n_params(d: int, W: int, L: int, bias: bool = True) -> int:
    """Number of learnable parameters of the MICNN (eq. icnn), with or without biases."""
    n = W * d + (L - 1) * (W * W + W * d) + W + d
    return n + (L * W if bias else 0)


def micnn_weights(rng: np.random.Generator, d: int, W: int, L: int, std: float = 0.1,
                  bias_std: float | None = None) -> dict:
    """Non-negative weights |N(0, std)| layer by layer; biases N(0, bias_std) or zero."""
    def nonneg(shape):
        return np.abs(rng.normal(0.0, std, size=shape))

    def bias(n):
        return rng.normal(0.0, bias_std, size=n) if bias_std else np.zeros(n)
    W1 = nonneg((W, d))
    c = np.zeros((L, W))
    c[0] = bias(W)
    Ak = np.zeros((max(L - 1, 0), W, W))
    Bk = np.zeros((max(L - 1, 0), W, d))
    for k in range(L - 1):
        Ak[k] = nonneg((W, W))
        Bk[k] = nonneg((W, d))
        c[k + 1] = bias(W)
    a = nonneg(W)
    b = nonneg(d)
    return dict(W1=W1, Ak=Ak, Bk=Bk, c=c, a=a, b=b)


def make_model(rng, kin: int, n_fib: int, W: int, L: int, kappa: float, std: float = 0.1,
               bias_std: float | None = None, stress_free: bool = False) -> ModelSpec:
    d = 3 + 2 * n_fib if kin == KIN_RAW else 3
    fib = FIBRES_PM30[:n_fib].copy() if n_fib else np.zeros((0, 3))
    w = micnn_weights(rng, d, W, L, std, bias_std)
    return ModelSpec(d=d, W=W, L=L, kin=kin, fibres=fib, kappa=kappa, stress_free=stress_free, **w)


# ----------------------------------------------------------------------- meshes

@dataclass
class Mesh:
    """Hex8 mesh: X[n_nodes][3] (float64), conn[n_el][8] (int32), nodes lexicographic."""
    X: np.ndarray
    conn: np.ndarray
    n: tuple

    @property
    def n_nodes(self) -> int:
        return int(self.X.shape[0])

    @property
    def n_el(self) -> int:
        return int(self.conn.shape[0])


def structured_mesh(nx: int, ny: int | None = None, nz: int | None = None,
                    lengths=(1.0, 1.0, 1.0)) -> Mesh:
    """Box [0,Lx]x[0,Ly]x[0,Lz] split into nx*ny*nz hex8 elements.

    Node (i, j, k) has index i + (nx+1) (j + (ny+1) k); element nodes follow the
    lexicographic reference order (x fastest), element (i, j, k) has index
    i + nx (j + ny k).
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    xs = np.linspace(0.0, lengths[0], nx + 1)
    ys = np.linspace(0.0, lengths[1], ny + 1)
    zs = np.linspace(0.0, lengths[2], nz + 1)
    Z, Y, Xc = np.meshgrid(zs, ys, xs, indexing="ij")
    X = np.stack([Xc.ravel(), Y.ravel(), Z.ravel()], axis=1)
    sx, sy = 1, nx + 1
    sz = (nx + 1) * (ny + 1)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    base = (i + sy * j + sz * k).ravel().astype(np.int64)
    offs = np.array([0, sx, sy, sx + sy, sz, sz + sx, sz + sy, sz + sx + sy], dtype=np.int64)
    conn = (base[:, None] + offs[None, :]).astype(np.int32)
    return Mesh(X=X, conn=conn, n=(nx, ny, nz))


def dof_count(nx: int, ny: int | None = None, nz: int | None = None) -> int:
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return 3 * (nx + 1) * (ny + 1) * (nz + 1)


# ------------------------------------------------------------ deformation inputs

def random_F(rng: np.random.Generator, n_qp: int, scale: float) -> np.ndarray:
    """F = I + scale*N(0,1) per entry per point, [n_qp][9]; points with det F <= 0 are
    redrawn in index order from the same stream until every det F > 0."""
    F = np.eye(3).ravel()[None, :] + scale * rng.normal(size=(n_qp, 9))
    while True:
        bad = np.nonzero(np.linalg.det(F.reshape(-1, 3, 3)) <= 0.0)[0]
        if bad.size == 0:
            return F
        F[bad] = np.eye(3).ravel()[None, :] + scale * rng.normal(size=(bad.size, 9))


def uniaxial_F(rng: np.random.Generator, n_qp: int, lo: float = 0.7, hi: float = 1.5,
               noise: float = 0.02) -> np.ndarray:
    """F = diag(lam, 1, 1) + noise*N(0,1), lam ~ U[lo, hi] per point, [n_qp][9]
    (the uniaxial-tension family of App. C with a perturbation); det F > 0 by redraw."""
    N = rng.normal(size=(n_qp, 9))
    lam = rng.uniform(lo, hi, size=n_qp)
    F = noise * N
    F[:, 0] += lam
    F[:, 4] += 1.0
    F[:, 8] += 1.0
    while True:
        bad = np.nonzero(np.linalg.det(F.reshape(-1, 3, 3)) <= 0.0)[0]
        if bad.size == 0:
            return F
        Nb = rng.normal(size=(bad.size, 9))
        lb = rng.uniform(lo, hi, size=bad.size)
        F[bad] = noise * Nb
        F[bad, 0] += lb
        F[bad, 4] += 1.0
        F[bad, 8] += 1.0


def nodal_noise(rng: np.random.Generator, mesh: Mesh, scale: float) -> np.ndarray:
    """u = scale*N(0,1) per nodal component, [n_nodes][3]."""
    return scale * rng.normal(size=(mesh.n_nodes, 3))


def cantilever_u(mesh: Mesh, seed: int, delta: float = 0.1, noise_h: float = 0.1) -> np.ndarray:
    """End-loaded cantilever along x on the unit cube, [n_nodes][3]:
    u_z = delta x^2 (3 - x) / 2, u_x = -(z - 1/2) du_z/dx, plus noise_h*h*N(0,1) per
    nodal component (h = element size along x) everywhere except the clamped face x = 0,
    where u = 0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x, z = mesh.X[:, 0], mesh.X[:, 2]
    uz = delta * x * x * (3.0 - x) / 2.0
    duz = delta * (6.0 * x - 3.0 * x * x) / 2.0
    u = np.zeros_like(mesh.X)
    u[:, 2] = uz
    u[:, 0] = -(z - 0.5) * duz
    h = 1.0 / mesh.n[0]
    u += noise_h * h * rng.normal(size=u.shape)
    u[x == 0.0] = 0.0
    return u


def loading_path(kind: str, gamma: float) -> np.ndarray:
    """Deformation gradients of the six loading paths of App. C (UT, UC, BT, BC, SS, PS), [9]."""
    g = gamma
    F = np.eye(3)
    if kind == "UT":
        F[0, 0] = 1 + g
    elif kind == "UC":
        F[0, 0] = 1 / (1 + g)
    elif kind == "BT":
        F[0, 0] = F[1, 1] = 1 + g
    elif kind == "BC":
        F[0, 0] = F[1, 1] = 1 / (1 + g)
    elif kind == "SS":
        F[0, 1] = g
    elif kind == "PS":
        F[0, 0] = 1 + g
        F[1, 1] = 1 / (1 + g)
    else:
        raise ValueError(kind)
    return F.ravel()


# ------------------------------------------------------------------- workloads

def workload_c0():
    """Plain FP64: 8^3 unit cube, 512 elements, 4096 qp; isotropic MICNN d3 W16 L2,
    kappa 10; u = 0.05 h N(0,1) per nodal component (h = 1/8, the element edge), seed 0.
    At this amplitude every Gauss point has det F > 0 (checked by the CPU tests)."""
    rng = np.random.Generator(np.random.PCG64(0))
    model = make_model(rng, KIN_ISO_SHIFTED, 0, W=16, L=2, kappa=10.0)
    mesh = structured_mesh(8)
    u = nodal_noise(rng, mesh, scale=0.05 / 8)
    return dict(name="c0_cube8_iso_d3w16l2", model=model, mesh=mesh, u=u)


# CANN term menus (eq. cann-fs): f0 in {x, <x>, |x|}, f1 = x^p, f2 in {w1 y, exp(w1 y) - 1, -ln(1 - w1 y)}
CANN_F0_ID, CANN_F0_MACAULAY, CANN_F0_ABS = 0, 1, 2
CANN_F2_LINEAR, CANN_F2_EXP, CANN_F2_LOG = 0, 1, 2
# the paper's CANN (App. C table): exponents {1, 2} x functions {x, exp(x)}
CANN_PAPER_KINDS = np.array([[CANN_F0_ID, 1, CANN_F2_LINEAR], [CANN_F0_ID, 1, CANN_F2_EXP],
                             [CANN_F0_ID, 2, CANN_F2_LINEAR], [CANN_F0_ID, 2, CANN_F2_EXP]], dtype=np.int32)


@dataclass
class CannSpec:
    """A CANN strain energy (eq. cann-def): n terms per input, kinds[n][3] = (f0, p, f2)
    shared by the inputs, weights w[d][n][2] = (w1, w2) per input and term."""
    d: int
    kin: int
    fibres: np.ndarray
    n: int
    kinds: np.ndarray
    w: np.ndarray
    kappa: float = 0.0
    stress_free: bool = False
    inner_name: str = "cann"

    def theta(self) -> np.ndarray:
        return np.asarray(self.w, dtype=np.float64).ravel().copy()


@dataclass
class GentThomasSpec:
    """The closed-form Gent-Thomas energy of eq. gt on raw (Ibar1, Ibar2, J); no parameters."""
    d: int = 3
    kin: int = KIN_RAW
    fibres: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    kappa: float = 0.0
    stress_free: bool = False
    inner_name: str = "gent_thomas"


@dataclass
class IckanSpec:
    """An input-convex KAN (App. B): widths [d, n_1, .., n_{R-1}, 1]; per layer r a uniform grid
    of G intervals on [lo[r], hi[r]] with B-splines of degree `degree` (knots extended by
    `degree` on each side, G + degree basis functions); params = per spline (layer, output i,
    input j order) the weight w_s then the control points."""
    d: int
    kin: int
    fibres: np.ndarray
    widths: list
    degree: int
    G: int
    lo: np.ndarray
    hi: np.ndarray
    params: np.ndarray
    kappa: float = 0.0
    stress_free: bool = False
    inner_name: str = "ickan"

    def theta(self) -> np.ndarray:
        return np.asarray(self.params, dtype=np.float64).copy()


def make_ickan(rng, kin: int = KIN_POLYCONVEX, widths=(3, 4, 4, 1), degree: int = 4, G: int = 30,
               lo0: float = -0.5, hi0: float = 12.0, kappa: float = 0.0) -> IckanSpec:
    """ICKAN with convex, non-decreasing splines (App. B condition c_{l+2} - c_{l+1} >=
    c_{l+1} - c_l >= 0: control points are cumulative sums of non-decreasing increments) and
    positive weights. Layer 0's grid is [lo0, hi0], wide enough for the kinematic scalars of
    F = I + 0.15 N(0,1) (outside its grid a KAN is neither monotone nor convex); each later
    layer's grid is the range its inputs can take (on its grid a spline lies between its first
    and last control point), with a 5 % margin."""
    widths = list(widths)
    d = widths[0]
    nb = G + degree
    lo, hi, params = [lo0], [hi0], []
    for r in range(len(widths) - 1):
        nin, nout = widths[r], widths[r + 1]
        zmin, zmax = np.zeros(nout), np.zeros(nout)
        for i in range(nout):
            for j in range(nin):
                w = 0.1 + abs(rng.normal(0.0, 0.5))
                inc = np.cumsum(np.abs(rng.normal(0.0, 0.1, size=nb - 1)))   # non-decreasing increments
                c = np.concatenate([[0.0], np.cumsum(inc)]) * (1.0 / max(1e-12, inc.sum()))
                params.append(np.concatenate([[w], c]))
                zmin[i] += w * c[0]
                zmax[i] += w * c[-1]
        if r + 1 < len(widths) - 1:
            span = zmax.max() - zmin.min()
            lo.append(zmin.min() - 0.05 * span)
            hi.append(zmax.max() + 0.05 * span)
    fib = np.zeros((0, 3))
    return IckanSpec(d=d, kin=kin, fibres=fib, widths=widths, degree=degree, G=G, lo=np.array(lo),
                     hi=np.array(hi), params=np.concatenate(params), kappa=kappa)


def workload_ickan(n: int = 64, seed: int = 8):
    """An ICKAN with the paper's spline settings (App. C: 2 hidden layers, order 4, 30 grid
    points; widths 3 -> 4 -> 4 -> 1) on the polyconvex inputs; F = I + 0.15 N(0,1), n^3 mesh."""
    rng = np.random.Generator(np.random.PCG64(seed))
    model = make_ickan(rng)
    mesh = structured_mesh(n)
    F = random_F(rng, 8 * mesh.n_el, 0.15)
    return dict(name=f"ickan_polyconvex_{n}cube_3x4x4x1_k4_g30", model=model, mesh=mesh, F=F)


def make_cann(rng, kin: int = KIN_POLYCONVEX, n_fib: int = 0, kinds=None, kappa: float = 0.0,
              std: float = 0.1, stress_free: bool = False) -> CannSpec:
    """CANN with |N(0, std)| weights drawn input by input, term by term (w1 then w2)."""
    kinds = CANN_PAPER_KINDS if kinds is None else np.asarray(kinds, dtype=np.int32)
    d = 3 + 2 * n_fib if kin == KIN_RAW else 3
    fib = FIBRES_PM30[:n_fib].copy() if n_fib else np.zeros((0, 3))
    w = np.abs(rng.normal(0.0, std, size=(d, kinds.shape[0], 2)))
    return CannSpec(d=d, kin=kin, fibres=fib, n=int(kinds.shape[0]), kinds=kinds, w=w, kappa=kappa,
                    stress_free=stress_free)


def workload_cann(n: int = 64, seed: int = 6):
    """The paper's CANN (App. C): exponents {1, 2} x {x, exp(x)} on the polyconvex inputs,
    24 weights; F = I + 0.15 N(0,1) on an n^3 mesh."""
    rng = np.random.Generator(np.random.PCG64(seed))
    model = make_cann(rng)
    mesh = structured_mesh(n)
    F = random_F(rng, 8 * mesh.n_el, 0.15)
    return dict(name=f"cann_polyconvex_{n}cube_4terms", model=model, mesh=mesh, F=F)


def workload_gent_thomas(n: int = 64, seed: int = 7):
    """The closed-form Gent-Thomas model of eq. gt (the paper's traditional-law comparison
    in its model-size study); F = I + 0.15 N(0,1) on an n^3 mesh."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mesh = structured_mesh(n)
    F = random_F(rng, 8 * mesh.n_el, 0.15)
    return dict(name=f"gent_thomas_{n}cube", model=GentThomasSpec(), mesh=mesh, F=F)


def twist_dirichlet(mesh, frac: float, stretch: float = 1.0, turns: float = 0.5):
    """Prescribed displacements of the twisting-cube benchmark (Sec. 4.3) at load fraction
    frac: the x = 0 face clamped; the x = Lx face moved frac * stretch along x and rotated by
    frac * turns * 2 pi about its centre line (y, z) = (Ly / 2, Lz / 2). Returns the fixed
    dofs (3 node + i, int64, sorted) and their displacement values."""
    X = np.asarray(mesh.X, dtype=np.float64)
    x0, x1 = X[:, 0].min(), X[:, 0].max()
    cy, cz = 0.5 * (X[:, 1].min() + X[:, 1].max()), 0.5 * (X[:, 2].min() + X[:, 2].max())
    left = np.nonzero(np.isclose(X[:, 0], x0))[0]
    right = np.nonzero(np.isclose(X[:, 0], x1))[0]
    th = frac * turns * 2.0 * math.pi
    c, s_ = math.cos(th), math.sin(th)
    yr, zr = X[right, 1] - cy, X[right, 2] - cz
    ur = np.stack([np.full(right.size, frac * stretch), c * yr - s_ * zr - yr, s_ * yr + c * zr - zr], axis=1)
    nodes = np.concatenate([left, right])
    vals = np.concatenate([np.zeros((left.size, 3)), ur])
    dofs = (3 * nodes[:, None] + np.arange(3)[None, :]).ravel()
    order = np.argsort(dofs, kind="stable")
    return dofs[order].astype(np.int64), vals.ravel()[order]


def workload_paper_ncm(n: int = 64, seed: int = 5):
    """The paper's NCM architecture (App. C, hyper-parameter table): MICNN with 3 hidden
    layers of 16 neurons, no biases (675 parameters), on the polyconvex kinematic layer
    K = (Ibar1 - 3, Ibar2^{3/2} - 3^{3/2}, (J - 1)^2); random non-negative weights (the
    trained weights do not ship); F = I + 0.15 N(0,1) per point on an n^3 mesh."""
    rng = np.random.Generator(np.random.PCG64(seed))
    model = make_model(rng, KIN_POLYCONVEX, 0, W=16, L=3, kappa=0.0)
    mesh = structured_mesh(n)
    F = random_F(rng, 8 * mesh.n_el, 0.15)
    return dict(name=f"ncm_polyconvex_{n}cube_d3w16l3", model=model, mesh=mesh, F=F)


def workload_c1(n: int = 64, seed: int = 1):
    """Anisotropic: n^3 hex8 mesh, 8 qp per element (element e owns qp 8e..8e+7);
    two fibres at +-30 deg; raw inputs (Ibar1, Ibar2, J, I4_11, I4_22, I5_11, I5_22);
    MICNN W32 L3, kappa 0; F = I + 0.15 N(0,1) per point."""
    rng = np.random.Generator(np.random.PCG64(seed))
    model = make_model(rng, KIN_RAW, 2, W=32, L=3, kappa=0.0)
    mesh = structured_mesh(n)
    F = random_F(rng, 8 * mesh.n_el, 0.15)
    return dict(name=f"c1_aniso_{n}cube_d7w32l3", model=model, mesh=mesh, F=F)


def workload_c2(n: int = 128, seed: int = 2):
    """Precision: n^3 mesh (8 n^3 qp); isotropic MICNN d3 W64 L3; uniaxial stretch
    lam in [0.7, 1.5] plus 0.02 N(0,1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    model = make_model(rng, KIN_ISO_SHIFTED, 0, W=64, L=3, kappa=10.0)
    mesh = structured_mesh(n)
    F = uniaxial_F(rng, 8 * mesh.n_el)
    return dict(name=f"c2_uniaxial_{n}cube_d3w64l3", model=model, mesh=mesh, F=F)


def workload_c3(n_qp: int = 1 << 20, seed: int = 3, inner: str = "micnn"):
    """Differentiation: the C1 network (seed 1 weights), n_qp points F = I + 0.15 N(0,1)
    drawn from seed 3; target model Neo-Hookean plus fibres (mu 1, k1 2, k2 0.5, kappa 10).
    inner = "cann": the same loss for the paper's CANN (App. C, the weights of
    workload_cann) on the same points; its target has no fibres (Neo-Hookean, kappa 10)."""
    model = workload_c1(n=1)["model"] if inner == "micnn" else workload_cann(n=1)["model"]
    rng = np.random.Generator(np.random.PCG64(seed))
    F = random_F(rng, n_qp, 0.15)
    target = dict(mu=1.0, k1=2.0, k2=0.5, kappa=10.0)
    tag = "d7w32l3" if inner == "micnn" else "cann_polyconvex_4terms"
    return dict(name=f"c3_backward_{n_qp}qp_{tag}", model=model, F=F, target=target)


def workload_residual(n: int = 64, seed: int = 9):
    """Gradient of a residual-based loss (eq. loss without reaction terms): the C1 network on an
    n^3 cantilever (the displacement field of c4, clamped at x = 0); L = 1/2 |r_free|^2, with
    the x = 0 dofs fixed."""
    model = workload_c1(n=1)["model"]
    mesh = structured_mesh(n)
    u = cantilever_u(mesh, seed)
    free = np.ones((mesh.n_nodes, 3))
    free[np.isclose(mesh.X[:, 0], 0.0)] = 0.0
    return dict(name=f"residual_loss_{n}cube_d7w32l3", model=model, mesh=mesh, u=u, free=free.ravel())


def workload_c4(n: int = 96, seed: int = 4):
    """Newton hot path: n^3 cantilever, anisotropic d7 W32 L3 network (C1 weights),
    end-load displacement field."""
    model = workload_c1(n=1)["model"]
    mesh = structured_mesh(n)
    u = cantilever_u(mesh, seed)
    return dict(name=f"c4_cantilever_{n}cube_d7w32l3", model=model, mesh=mesh, u=u)
