"""Seeded synthetic problem descriptions (inputs only -- no ADMM arithmetic).

Both the CUDA path (through the C-ABI binding) and the FP64 oracle consume
the same ``Problem`` objects built here; this module holds no proximal
operator, no update rule and no residual.  Every generator is deterministic
in its seed.

Workloads (paper Sec. V):
  * circle packing in a triangle (Sec. V-A, Appendix A): N disks, pairwise
    no-overlap factors, one wall factor per disk and triangle side, one
    radius-reward factor per disk; 2N variable nodes (c_i in R^2, r_i);
    2N^2 - N + 2NS edges; N(N-1)/2 + N + NS factors.
  * linear soft-margin SVM (Sec. V-C): one hinge factor per point on a
    shared (w, b) plus an L2 factor on w; or the paper's own form, a copy
    of w per point with margin, slack, split-norm and equality factors.
  * linear MPC (Sec. V-B, Appendix B): states x_0..x_T, inputs u_0..u_{T-1};
    a fixed-x_0 factor, dynamics, diagonal quadratic costs and input boxes;
    batches of small instances, or one inverted-pendulum instance with a
    horizon of up to 10^5 steps.
"""
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

# Factor types: the interface numbers of the C-ABI (include/fgadmm.h).
PACK_PAIR = 0
PACK_WALL = 1
PACK_RADIUS_LIN = 2
PACK_RADIUS_QUAD = 3
SVM_HINGE = 4
SVM_L2 = 5
MPC_DYN = 6
MPC_QUAD = 7
MPC_BOX = 8
FIX = 9
SVM_MARGIN = 10
SVM_SLACK = 11
EQUAL = 12


@dataclass
class FactorBlock:
    ftype: int
    var_ids: np.ndarray          # (count, nv) int64
    params: np.ndarray           # (count, np) float64, np may be 0


@dataclass
class Problem:
    """A factor graph: variable blocks, factor blocks (both in creation
    order), a start point z0 (scalar variables, variable order) and uniform
    rho/alpha."""
    name: str
    var_blocks: List[Tuple[int, int]] = field(default_factory=list)   # (count, dim)
    factor_blocks: List[FactorBlock] = field(default_factory=list)
    z0: Optional[np.ndarray] = None
    rho: float = 1.0
    alpha: float = 1.0
    meta: dict = field(default_factory=dict)

    def add_vars(self, count, dim):
        first = sum(c for c, _ in self.var_blocks)
        self.var_blocks.append((int(count), int(dim)))
        return first

    def add_factors(self, ftype, var_ids, params=None):
        var_ids = np.ascontiguousarray(np.asarray(var_ids, dtype=np.int64))
        if var_ids.ndim == 1:
            var_ids = var_ids[None, :]
        count = var_ids.shape[0]
        if params is None:
            params = np.zeros((count, 0))
        params = np.asarray(params, dtype=np.float64)
        if params.ndim == 1:
            params = np.broadcast_to(params, (count, params.shape[0]))
        self.factor_blocks.append(FactorBlock(int(ftype), var_ids, np.ascontiguousarray(params)))

    # sizes -----------------------------------------------------------------
    def var_dims(self):
        return np.concatenate([np.full(c, d, dtype=np.int64) for c, d in self.var_blocks]) \
            if self.var_blocks else np.zeros(0, np.int64)

    @property
    def num_vars(self):
        return sum(c for c, _ in self.var_blocks)

    @property
    def num_scalar_vars(self):
        return sum(c * d for c, d in self.var_blocks)

    @property
    def num_factors(self):
        return sum(b.var_ids.shape[0] for b in self.factor_blocks)

    @property
    def num_edges(self):
        dims = self.var_dims()
        return int(sum(dims[b.var_ids].sum() for b in self.factor_blocks))


# ---------------------------------------------------------------------------
# Circle packing in an equilateral triangle of side 1 (Sec. V-A).
# ---------------------------------------------------------------------------

TRIANGLE = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, np.sqrt(3.0) / 2.0]])


def triangle_walls():
    """Unit inward normals Q_s and a point V_s on each side s = 1, 2, 3."""
    s3 = np.sqrt(3.0) / 2.0
    Q = np.array([[0.0, 1.0], [s3, -0.5], [-s3, -0.5]])
    V = np.array([[0.0, 0.0], [0.0, 0.0], [1.0, 0.0]])
    return Q, V


def packing_start(N, seed):
    """Centres uniform in the triangle (two uniforms, reflected when their
    sum exceeds 1), radii uniform in [0, 0.05]."""
    rng = np.random.default_rng(seed)
    a = rng.random((N, 2))
    flip = a.sum(axis=1) > 1.0
    a[flip] = 1.0 - a[flip]
    P0, P1, P2 = TRIANGLE
    c = P0 + a[:, :1] * (P1 - P0) + a[:, 1:] * (P2 - P0)
    r = rng.random(N) * 0.05
    return c, r


def packing_problem(N, seed=1000, reward="lin", rho=1.0, alpha=1.0):
    """N disks in the unit triangle.  Variables, in creation order:
    c_0, r_0, c_1, r_1, ...  Factors: all pairs (i < j, row-major), then
    walls (disk-major, sides 1..3), then one radius reward per disk."""
    p = Problem("packing_N%d" % N, rho=rho, alpha=alpha)
    p.var_blocks = [(1, 2), (1, 1)] * N
    cid = 2 * np.arange(N, dtype=np.int64)
    rid = cid + 1
    if N >= 2:
        i, j = np.triu_indices(N, k=1)
        pairs = np.stack([cid[i], rid[i], cid[j], rid[j]], axis=1)
        p.add_factors(PACK_PAIR, pairs)
    Q, V = triangle_walls()
    wv = np.repeat(np.stack([cid, rid], axis=1), 3, axis=0)
    wp = np.tile(np.concatenate([Q, V], axis=1), (N, 1))
    p.add_factors(PACK_WALL, wv, wp)
    if reward == "lin":
        p.add_factors(PACK_RADIUS_LIN, rid[:, None], np.ones((N, 1)))
    elif reward == "quad":
        p.add_factors(PACK_RADIUS_QUAD, rid[:, None])
    else:
        raise ValueError(reward)
    c, r = packing_start(N, seed)
    z0 = np.empty(3 * N)
    z0[0::3] = c[:, 0]
    z0[1::3] = c[:, 1]
    z0[2::3] = r
    p.z0 = z0
    p.meta = dict(N=N, S=3, seed=seed)
    return p


def packing_counts(N, S=3):
    """Edge / variable-node / factor counts stated in Sec. V-A."""
    return dict(edges=2 * N * N - N + 2 * N * S, var_nodes=2 * N,
                factors=N * (N - 1) // 2 + N + N * S)


# ---------------------------------------------------------------------------
# Linear soft-margin SVM (Sec. V-C, hinge form on a shared (w, b)).
# ---------------------------------------------------------------------------

def svm_data(npts, d, seed, sep=0.5, flip=0.05):
    """Two isotropic unit-variance Gaussians with means +-sep*1, labels +-1,
    a fraction `flip` of labels flipped."""
    rng = np.random.default_rng(seed)
    y = np.where(np.arange(npts) % 2 == 0, 1.0, -1.0)
    rng.shuffle(y)
    X = rng.standard_normal((npts, d)) + sep * y[:, None]
    nflip = int(round(flip * npts))
    idx = rng.choice(npts, size=nflip, replace=False)
    y = y.copy()
    y[idx] = -y[idx]
    return X, y


def svm_problem(npts, d, seed=3000, lam=1e-3, c=1.0, rho=1.0, alpha=1.0, X=None, y=None):
    """Variables w (dim d), b (dim 1); one hinge factor per point, then one
    L2 factor (lambda/2)|w|^2."""
    if X is None:
        X, y = svm_data(npts, d, seed)
    p = Problem("svm_%dx%d" % (npts, d), rho=rho, alpha=alpha)
    w = p.add_vars(1, d)
    b = p.add_vars(1, 1)
    vids = np.tile(np.array([w, b], dtype=np.int64), (npts, 1))
    params = np.concatenate([X, y[:, None], np.full((npts, 1), c)], axis=1)
    p.add_factors(SVM_HINGE, vids, params)
    p.add_factors(SVM_L2, np.array([[w]]), np.array([[lam]]))
    p.z0 = np.zeros(d + 1)
    p.meta = dict(X=X, y=y, lam=lam, c=c)
    return p


def svm_paper_problem(npts, d, seed=3000, C=1000.0, rho=1.0, alpha=1.0, X=None, y=None):
    """The soft-margin SVM in the paper's own factor-graph form (Sec. V-C,
    Appendix C): min 1/2 |w|^2 + C sum xi_i subject to y_i (w.x_i + b) >=
    1 - xi_i, xi_i >= 0, with one copy w_i of w per point and the norm term
    split into N equal parts.  Variables in creation order: the copies
    w_1..w_N (one block of dimension d), b, the slacks xi_1..xi_N.  Factors:
    one margin factor per point on (w_i, b, xi_i); one minimal-error factor
    per slack (weight C); one norm factor (1/(2N)) |w_i|^2 per copy; the
    equality factors w_i = w_{i+1}, i = 1..N-1, a chain.  The same minimiser
    (w, b) as svm_problem with c = C, lam = 1, or c = 1, lam = 1/C."""
    if X is None:
        X, y = svm_data(npts, d, seed)
    p = Problem("svm_paper_%dx%d" % (npts, d), rho=rho, alpha=alpha)
    w0 = p.add_vars(npts, d)
    b = p.add_vars(1, 1)
    xi0 = p.add_vars(npts, 1)
    ws = w0 + np.arange(npts, dtype=np.int64)
    xis = xi0 + np.arange(npts, dtype=np.int64)
    p.add_factors(SVM_MARGIN, np.stack([ws, np.full(npts, b, dtype=np.int64), xis], axis=1),
                  np.concatenate([X, y[:, None]], axis=1))
    p.add_factors(SVM_SLACK, xis[:, None], np.array([C]))
    p.add_factors(SVM_L2, ws[:, None], np.array([1.0 / npts]))
    if npts > 1:
        p.add_factors(EQUAL, np.stack([ws[:-1], ws[1:]], axis=1))
    p.z0 = np.zeros(p.num_scalar_vars)
    p.meta = dict(X=X, y=y, C=C, w0=w0, b=b, xi0=xi0)
    return p


def svm_paper_edges(npts, d):
    """Scalar edges of svm_paper_problem: margins N(d + 2), slacks N, norms
    N d, equalities 2 d (N - 1)."""
    return npts * (d + 2) + npts + npts * d + 2 * d * max(npts - 1, 0)


# ---------------------------------------------------------------------------
# Linear MPC (Sec. V-B, Appendix B), x_{t+1} = A x_t + B u_t.
# ---------------------------------------------------------------------------

def mpc_system(nx, nu, rng, spectral_radius=0.95):
    """A = 0.95 G / rho(G) with G standard normal; B Gaussian / sqrt(nx);
    Q, R diagonal from U[0.1, 10]."""
    G = rng.standard_normal((nx, nx))
    A = spectral_radius * G / np.max(np.abs(np.linalg.eigvals(G)))
    B = rng.standard_normal((nx, nu)) / np.sqrt(nx)
    q = rng.uniform(0.1, 10.0, nx)
    r = rng.uniform(0.1, 10.0, nu)
    return A, B, q, r


def mpc_batch_inputs(n_inst, seed=4000, nx=12, nu=4, tmin=10, tmax=50, shared_system=False,
                     T_fixed=None, umax=1.0):
    """Ragged batch of MPC instances: horizons uniform on {tmin..tmax} (or
    T_fixed), one system per instance (or one shared system), x0 ~ N(0, I)."""
    rng = np.random.default_rng(seed)
    if T_fixed is not None:
        T = np.full(n_inst, int(T_fixed), dtype=np.int32)
    else:
        T = rng.integers(tmin, tmax + 1, size=n_inst).astype(np.int32)
    if shared_system:
        A, B, q, r = mpc_system(nx, nu, rng)
        A = A[None]; B = B[None]; q = q[None]; r = r[None]
    else:
        sys = [mpc_system(nx, nu, rng) for _ in range(n_inst)]
        A = np.stack([s[0] for s in sys]); B = np.stack([s[1] for s in sys])
        q = np.stack([s[2] for s in sys]); r = np.stack([s[3] for s in sys])
    x0 = rng.standard_normal((n_inst, nx))
    return dict(T=T, A=A, B=B, q=q, r=r, x0=x0, nx=nx, nu=nu, umax=float(umax),
                shared_system=bool(shared_system))


def mpc_warmstart_inputs(n_inst, system_seed=5000, x0_seed=5001, T=30, nx=12, nu=4, umax=1.0):
    """Learned-warm-start workload: ONE fixed system of the MPC family (drawn
    with system_seed) and n_inst initial states x0 ~ N(0, I) (x0_seed), all
    with horizon T.  Training and evaluation sets use different x0 seeds."""
    A, B, q, r = mpc_system(nx, nu, np.random.default_rng(system_seed))
    x0 = np.random.default_rng(x0_seed).standard_normal((n_inst, nx))
    return dict(T=np.full(n_inst, T, dtype=np.int32), A=A[None], B=B[None], q=q[None], r=r[None], x0=x0,
                nx=nx, nu=nu, umax=float(umax), shared_system=True)


def mpc_problem(A, B, q, r, x0, T, umax=1.0, rho=1.0, alpha=1.0):
    """One MPC instance as a general factor graph.  Variables in creation
    order: x_0, u_0, x_1, u_1, ..., u_{T-1}, x_T.  Factors: FIX(x_0);
    DYN(x_t, u_t, x_{t+1}) t = 0..T-1; stage QUAD(x_t, u_t) with diag(q, r);
    terminal QUAD(x_T) with diag(q); BOX(u_t) with [-umax, umax]."""
    nx, nu = B.shape
    p = Problem("mpc_T%d" % T, rho=rho, alpha=alpha)
    xs, us = [], []
    for t in range(T):
        xs.append(p.add_vars(1, nx))
        us.append(p.add_vars(1, nu))
    xs.append(p.add_vars(1, nx))
    xs = np.array(xs, dtype=np.int64)
    us = np.array(us, dtype=np.int64)
    p.add_factors(FIX, xs[:1, None], np.asarray(x0, dtype=np.float64)[None, :])
    dyn_params = np.concatenate([A.reshape(-1), B.reshape(-1)])
    p.add_factors(MPC_DYN, np.stack([xs[:-1], us, xs[1:]], axis=1), dyn_params)
    p.add_factors(MPC_QUAD, np.stack([xs[:-1], us], axis=1), np.concatenate([q, r]))
    p.add_factors(MPC_QUAD, xs[-1:, None], q)
    p.add_factors(MPC_BOX, us[:, None], np.array([-umax, umax]))
    p.z0 = np.zeros(p.num_scalar_vars)
    p.meta = dict(nx=nx, nu=nu, T=T, xs=xs, us=us)
    return p


def pendulum_system(dt=0.04, M=1.0, m=0.1, l=0.5, g=9.81):
    """The cart-and-pole inverted pendulum of Sec. V-B, linearised about the
    upright equilibrium and sampled every dt seconds with a zero-order hold.
    State (cart position, cart velocity, pole angle, angular velocity), input
    the force on the cart; cart mass M, a point mass m at distance l on a
    massless pole, no friction:
        p'' = (F - m g th) / M,    th'' = ((M + m) g th - F) / (M l).
    Returns (A_d, B_d) with x_{t+1} = A_d x_t + B_d u_t, i.e. the paper's
    q(t+1) - q(t) = A q(t) + B u(t) with A = A_d - I, B = B_d."""
    from scipy.linalg import expm
    Ac = np.zeros((4, 4))
    Ac[0, 1] = 1.0
    Ac[1, 2] = -m * g / M
    Ac[2, 3] = 1.0
    Ac[3, 2] = (M + m) * g / (M * l)
    Bc = np.array([[0.0], [1.0 / M], [0.0], [-1.0 / (M * l)]])
    aug = np.zeros((5, 5))
    aug[:4, :4] = Ac
    aug[:4, 4:] = Bc
    E = expm(aug * dt)
    return E[:4, :4].copy(), E[:4, 4:].copy()


def mpc_horizon_problem(K, seed=6000, q=(1.0, 0.1, 10.0, 0.1), r=(0.1,), umax=None, rho=1.0, alpha=1.0,
                        system=None):
    """One long-horizon MPC of the inverted pendulum (Sec. V-B: A 4 x 4,
    B 4 x 1, sampled at 40 ms, equal diagonal Q_t and R_t, horizon K from 200
    to 10^5) as a single factor graph.  Variables in creation order: the
    states x_0..x_K (one block of dimension 4), then the inputs
    u_0..u_{K-1} (one block of dimension 1).  Factors: FIX(x_0), DYN(x_t,
    u_t, x_{t+1}) t = 0..K-1, stage QUAD(x_t, u_t) with diag(q, r), terminal
    QUAD(x_K) with diag(q) (Q_f = Q), and BOX(u_t) only when umax is given.
    x_0 ~ N(0, diag(0.1, 0.1, 0.05, 0.1)^2) from the seed; z0 = 0."""
    A, B = pendulum_system() if system is None else system
    nx, nu = B.shape
    q = np.asarray(q, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    rng = np.random.default_rng(seed)
    x0 = rng.standard_normal(nx) * np.array([0.1, 0.1, 0.05, 0.1])[:nx]
    p = Problem("mpc_horizon_K%d" % K, rho=rho, alpha=alpha)
    x_first = p.add_vars(K + 1, nx)
    u_first = p.add_vars(K, nu)
    xs = x_first + np.arange(K + 1, dtype=np.int64)
    us = u_first + np.arange(K, dtype=np.int64)
    p.add_factors(FIX, xs[:1, None], x0[None, :])
    p.add_factors(MPC_DYN, np.stack([xs[:-1], us, xs[1:]], axis=1),
                  np.concatenate([A.reshape(-1), B.reshape(-1)]))
    p.add_factors(MPC_QUAD, np.stack([xs[:-1], us], axis=1), np.concatenate([q, r]))
    p.add_factors(MPC_QUAD, xs[-1:, None], q)
    if umax is not None:
        p.add_factors(MPC_BOX, us[:, None], np.array([-umax, umax]))
    p.z0 = np.zeros(p.num_scalar_vars)
    p.meta = dict(nx=nx, nu=nu, K=K, A=A, B=B, q=q, r=r, x0=x0, umax=umax)
    return p


def mpc_horizon_split(z, K, nx=4, nu=1):
    """(states (K+1, nx), inputs (K, nu)) of a mpc_horizon_problem solution
    in variable order."""
    z = np.asarray(z)
    return z[:(K + 1) * nx].reshape(K + 1, nx), z[(K + 1) * nx:].reshape(K, nu)


def mpc_horizon_edges(K, nx=4, nu=1, box=False):
    """Scalar edges of mpc_horizon_problem: FIX + K DYN + K stage + terminal
    (+ K BOX)."""
    return nx + (2 * nx + nu) * K + (nx + nu) * K + nx + (nu * K if box else 0)


def mpc_edges(T, nx=12, nu=4):
    """Scalar edges of one instance: FIX + T DYN + T stage + terminal + T BOX."""
    return nx + (2 * nx + nu) * T + (nx + nu) * T + nx + nu * T


def fig1_problem():
    """The Sec. II example f1(w1,w2,w3) + f2(w1,w4,w5) + f3(w2,w5) + f4(w5)
    with scalar variables, built from diagonal quadratic factors."""
    p = Problem("fig1")
    p.add_vars(5, 1)
    p.add_factors(MPC_QUAD, [[0, 1, 2]], [[1.0, 2.0, 3.0]])
    p.add_factors(MPC_QUAD, [[0, 3, 4]], [[1.5, 2.5, 0.5]])
    p.add_factors(MPC_QUAD, [[1, 4]], [[1.0, 1.0]])
    p.add_factors(MPC_QUAD, [[4]], [[2.0]])
    p.z0 = np.arange(1.0, 6.0)
    return p
