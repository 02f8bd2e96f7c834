"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds problem set-ups only: Cartesian mesh connectivity, initial
conditions written as functions of position, and random admissible states.  It
holds none of the limiter's or the FR scheme's arithmetic; in particular the
reference-element node positions are always passed in by the caller, so each
side (the CUDA library or the CPU checker) supplies its own.

Layouts: solution ``w[nv][E][Ns]`` with Ns = (p+1)^d nodes per element, x index
fastest; ``nbr[E][2d]`` faces ordered (-x, +x, -y, +y); a negative ``nbr`` is a
boundary face whose exterior state is ``bc[-(nbr+1)]``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 1.4


def conservative(rho, u, p, gamma=GAMMA):
    """(rho, u[d], P) -> (rho, rho u[d], P/(gamma-1) + rho |u|^2 / 2); u is a list of arrays."""
    rho = np.asarray(rho, dtype=np.float64)
    mom = [rho * np.asarray(ui, dtype=np.float64) for ui in u]
    ke = 0.5 * rho * sum(np.asarray(ui, dtype=np.float64) ** 2 for ui in u)
    return np.stack([rho, *mom, np.asarray(p, dtype=np.float64) / (gamma - 1.0) + ke])


@dataclass
class CartMesh:
    dim: int
    n: tuple            # elements per axis
    lo: tuple           # domain lower corner
    hi: tuple           # domain upper corner
    nbr: np.ndarray     # [E][2d] int32
    h: np.ndarray       # [E][d]
    centers: np.ndarray  # [E][d]
    bc: np.ndarray = field(default_factory=lambda: np.zeros((1, 4)))

    @property
    def n_elem(self):
        return self.nbr.shape[0]


def mesh_1d(n, x0, x1, periodic=False, bc_left=0, bc_right=1):
    """Uniform line mesh; boundary faces get ids bc_left / bc_right unless periodic."""
    e = np.arange(n)
    nbr = np.stack([e - 1, e + 1], axis=1).astype(np.int32)
    if periodic:
        nbr[0, 0], nbr[-1, 1] = n - 1, 0
    else:
        nbr[0, 0], nbr[-1, 1] = -(bc_left + 1), -(bc_right + 1)
    hx = (x1 - x0) / n
    h = np.full((n, 1), hx)
    centers = (x0 + (e + 0.5) * hx)[:, None]
    return CartMesh(1, (n,), (x0,), (x1,), nbr, h, centers)


def mesh_2d(nx, ny, x0, x1, y0, y1, periodic=(False, False), bc_of_face=None):
    """Uniform quad mesh, element e = iy * nx + ix.

    ``bc_of_face(ix, iy, f)`` gives the boundary ids of face f for arrays of element
    positions (default 0).
    """
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    ix, iy = ix.ravel(), iy.ravel()
    E = nx * ny
    nbr = np.zeros((E, 4), dtype=np.int64)
    for f, (dx, dy) in enumerate(((-1, 0), (1, 0), (0, -1), (0, 1))):
        jx, jy = ix + dx, iy + dy
        if periodic[0]:
            jx = jx % nx
        if periodic[1]:
            jy = jy % ny
        inside = (jx >= 0) & (jx < nx) & (jy >= 0) & (jy < ny)
        nb = np.where(inside, jy * nx + jx, 0)
        if bc_of_face is None:
            ids = np.zeros(E, dtype=np.int64)
        else:   # vectorised over elements
            ids = np.broadcast_to(np.asarray(bc_of_face(ix, iy, f), dtype=np.int64), (E,))
        nbr[:, f] = np.where(inside, nb, -(ids + 1))
    hx, hy = (x1 - x0) / nx, (y1 - y0) / ny
    h = np.tile([hx, hy], (E, 1)).astype(np.float64)
    centers = np.stack([x0 + (ix + 0.5) * hx, y0 + (iy + 0.5) * hy], axis=1)
    return CartMesh(2, (nx, ny), (x0, y0), (x1, y1), nbr.astype(np.int32), h, centers)


def node_coords(mesh: CartMesh, xi):
    """Physical coordinates of the solution nodes; xi are the 1D reference nodes on [-1, 1]."""
    xi = np.asarray(xi, dtype=np.float64)
    if mesh.dim == 1:
        x = mesh.centers[:, 0:1] + 0.5 * mesh.h[:, 0:1] * xi[None, :]
        return (x,)
    n = len(xi)
    X = np.tile(xi, n)          # i fastest
    Y = np.repeat(xi, n)
    x = mesh.centers[:, 0:1] + 0.5 * mesh.h[:, 0:1] * X[None, :]
    y = mesh.centers[:, 1:2] + 0.5 * mesh.h[:, 1:2] * Y[None, :]
    return x, y


# ---------------------------------------------------------------------------
# Problem set-ups
# ---------------------------------------------------------------------------
def sod(n=200, gamma=GAMMA):
    """Sod shock tube on [0, 1] (Sec. 6.1): (1, 0, 1) left of 0.5, (0.125, 0, 0.1) right."""
    mesh = mesh_1d(n, 0.0, 1.0, periodic=False, bc_left=0, bc_right=1)
    left = conservative(1.0, [0.0], 1.0, gamma)
    right = conservative(0.125, [0.0], 0.1, gamma)
    mesh.bc = np.stack([left, right]).astype(np.float64)

    def ic(x):
        return np.where(x <= 0.5, left[:, None, None], right[:, None, None])
    return mesh, ic


def riemann_1d(n, left, right, x0, x1, xs, gamma=GAMMA):
    """1D Riemann problem on [x0, x1]: primitive (rho, u, P) states left / right of xs, Dirichlet
    ends carrying the two states."""
    mesh = mesh_1d(n, x0, x1, periodic=False, bc_left=0, bc_right=1)
    ql = conservative(left[0], [left[1]], left[2], gamma)
    qr = conservative(right[0], [right[1]], right[2], gamma)
    mesh.bc = np.stack([ql, qr]).astype(np.float64)

    def ic(x):
        return np.where(x <= xs, ql[:, None, None], qr[:, None, None])
    return mesh, ic


def problem_123(n=100, gamma=GAMMA):
    """Double rarefaction ("123 problem", Sec. 6.3): [0, 1], (1, -2, 0.4) | (1, 2, 0.4) at x = 0.5."""
    return riemann_1d(n, (1.0, -2.0, 0.4), (1.0, 2.0, 0.4), 0.0, 1.0, 0.5, gamma)


LEBLANC_GAMMA = 5.0 / 3.0


def leblanc(n=100, gamma=LEBLANC_GAMMA):
    """Leblanc shock tube (Sec. 6.5): [0, 9], (1, 0, (gamma-1) 1e-1) | (1e-3, 0, (gamma-1) 1e-10) at
    x = 3.  The paper does not restate gamma here; the problem's usual value 5/3 is taken."""
    return riemann_1d(n, (1.0, 0.0, (gamma - 1) * 1e-1), (1e-3, 0.0, (gamma - 1) * 1e-10), 0.0, 9.0, 3.0, gamma)


def density_pulse(n, gamma=GAMMA, sigma=200.0):
    """Smooth convecting pulse on periodic [-0.5, 0.5] (Sec. 6.2): rho = 1 + exp(-sigma x^2), u = 1, P = 1.

    Sec. 6.2 prints sigma = 500, but its own error tables (Tables 3 and 4) are those of sigma = 200:
    an independent discontinuous Galerkin solution and the checker reproduce them to four digits
    with 200 and are five to twelve times larger with 500.  200 is taken."""
    mesh = mesh_1d(n, -0.5, 0.5, periodic=True)

    def ic(x, t=0.0):
        xs = (x - t + 0.5) % 1.0 - 0.5
        return conservative(1.0 + np.exp(-sigma * xs * xs), [np.ones_like(xs)], np.ones_like(xs), gamma)
    return mesh, ic


def isentropic_vortex(n=128, gamma=GAMMA, beta=5.0, L=10.0, u0=1.0, v0=1.0):
    """Isentropic vortex on periodic [0, L]^2, mean flow (u0, v0), strength beta, centre (L/2, L/2).

    Velocity perturbation beta/(2 pi) exp((1 - r^2)/2) (-(y-yc), x-xc); temperature
    T = 1 - (gamma-1) beta^2 / (8 gamma pi^2) exp(1 - r^2); rho = T^(1/(gamma-1)), P = rho^gamma.
    The exact solution is the initial field translated by (u0, v0) t.
    """
    mesh = mesh_2d(n, n, 0.0, L, 0.0, L, periodic=(True, True))

    def ic(x, y, t=0.0):
        xc = (x - u0 * t) % L - L / 2
        yc = (y - v0 * t) % L - L / 2
        r2 = xc * xc + yc * yc
        a = beta / (2 * math.pi) * np.exp(0.5 * (1 - r2))
        T = 1 - (gamma - 1) * beta * beta / (8 * gamma * math.pi ** 2) * np.exp(1 - r2)
        rho = T ** (1 / (gamma - 1))
        return conservative(rho, [u0 - a * yc, v0 + a * xc], rho ** gamma, gamma)
    return mesh, ic


def sedov(n=512, gamma=GAMMA, rho0=1.0, p_amb=1e-6, e_total=1.0, L=1.2):
    """Sedov-type blast on [-L, L]^2 (Sec. 6.6 layout): ambient (rho0, 0, p_amb), total energy
    e_total deposited uniformly in the four elements touching the centre (n must be even)."""
    assert n % 2 == 0
    mesh = mesh_2d(n, n, -L, L, -L, L)
    amb = conservative(rho0, [0.0, 0.0], p_amb, gamma)
    mesh.bc = amb[None, :].astype(np.float64)
    hx = 2 * L / n
    p_c = (gamma - 1) * (e_total / 4) / (hx * hx)
    centre = np.zeros(mesh.n_elem, dtype=bool)
    c0 = n // 2 - 1
    for iy in (c0, c0 + 1):
        for ix in (c0, c0 + 1):
            centre[iy * n + ix] = True

    def ic(x, y):
        w = np.broadcast_to(amb[:, None, None], (4,) + x.shape).copy()
        hot = conservative(rho0, [0.0, 0.0], p_c, gamma)
        w[:, centre, :] = hot[:, None, None]
        return w
    return mesh, ic


def four_quadrant_states(rng, gamma=GAMMA):
    """Four quadrant states (rho, u, v, P) with rho, P ~ U[0.1, 2], u, v ~ U[-1, 1]; order
    (x<0.5,y<0.5), (x>=0.5,y<0.5), (x<0.5,y>=0.5), (x>=0.5,y>=0.5)."""
    rho = rng.uniform(0.1, 2.0, 4)
    P = rng.uniform(0.1, 2.0, 4)
    u = rng.uniform(-1.0, 1.0, 4)
    v = rng.uniform(-1.0, 1.0, 4)
    return conservative(rho, [u, v], P, gamma).T.copy()   # [4][nv]


def four_quadrant(n, states):
    """One four-quadrant Riemann problem on [0, 1]^2 with n x n elements; each boundary face
    takes the state of the quadrant it lies in (Dirichlet)."""
    def q(ix, iy, f=None):
        return (ix >= n // 2).astype(int) + 2 * (iy >= n // 2).astype(int)
    mesh = mesh_2d(n, n, 0.0, 1.0, 0.0, 1.0, bc_of_face=q)
    mesh.bc = np.asarray(states, dtype=np.float64)

    def ic(x, y):
        qi = (x >= 0.5).astype(int) + 2 * (y >= 0.5).astype(int)
        return np.asarray(states).T[:, qi]
    return mesh, ic


def shock_vortex(n, gamma=GAMMA, mach=1.1, beta=1.0, radius=0.1, centre=(0.25, 0.5), shock_x=0.5):
    """Shock-vortex interaction on [0, 2] x [0, 1] with n x n elements (n a multiple of 4, so that
    x = shock_x = 0.5 is an element boundary): a stationary normal shock between the upstream
    state (rho, u, v, P) = (1, mach sqrt(gamma), 0, 1) and its Rankine-Hugoniot post-shock state,
    and an isentropic vortex of strength beta and core radius `radius` centred upstream at
    `centre`, carried into the shock by the mean flow.  x faces take the upstream (left) and
    post-shock (right) states; y is periodic.

    Vortex (the form of the isentropic-vortex set-up, lengths in units of `radius`), with
    r = |x - centre| / radius: velocity perturbation beta/(2 pi) exp((1 - r^2)/2) (-(y-yc), x-xc)
    / radius; temperature T = 1 - (gamma-1) beta^2 / (8 gamma pi^2) exp(1 - r^2);
    rho = T^(1/(gamma-1)), P = rho^gamma.  With beta = 1 the peak swirl speed is 0.26, a vortex
    Mach number of about 0.22.
    """
    assert n % 4 == 0
    m2 = mach * mach
    c1 = math.sqrt(gamma)
    u1 = mach * c1
    rho2 = (gamma + 1) * m2 / ((gamma - 1) * m2 + 2)
    p2 = 1 + 2 * gamma / (gamma + 1) * (m2 - 1)
    u2 = u1 / rho2
    up = conservative(1.0, [u1, 0.0], 1.0, gamma)
    down = conservative(rho2, [u2, 0.0], p2, gamma)

    def bc_of_face(ix, iy, f):
        return np.full(np.shape(ix), 0 if f == 0 else 1)
    mesh = mesh_2d(n, n, 0.0, 2.0, 0.0, 1.0, periodic=(False, True), bc_of_face=bc_of_face)
    mesh.bc = np.stack([up, down]).astype(np.float64)

    def ic(x, y):
        xc = (x - centre[0]) / radius
        yc = (y - centre[1]) / radius
        r2 = xc * xc + yc * yc
        a = beta / (2 * math.pi) * np.exp(0.5 * (1 - r2))
        T = 1 - (gamma - 1) * beta * beta / (8 * gamma * math.pi ** 2) * np.exp(1 - r2)
        rho = T ** (1 / (gamma - 1))
        vort = conservative(rho, [u1 - a * yc, a * xc], rho ** gamma, gamma)
        post = np.broadcast_to(down.reshape((4,) + (1,) * x.ndim), vort.shape)
        return np.where(x[None] < shock_x, vort, post)
    return mesh, ic


def nodal_field(mesh: CartMesh, xi, ic):
    """w[nv][E][Ns] = ic evaluated at the solution nodes built from reference nodes xi."""
    return np.ascontiguousarray(ic(*node_coords(mesh, xi)), dtype=np.float64)


# ---------------------------------------------------------------------------
# Random admissible data
# ---------------------------------------------------------------------------
def random_states(rng, n, dim, rho=(0.1, 2.0), vel=(-1.0, 1.0), p=(0.1, 2.0), gamma=GAMMA):
    """n random admissible conservative states, shape [n][d+2]."""
    r = rng.uniform(*rho, n)
    u = [rng.uniform(*vel, n) for _ in range(dim)]
    P = rng.uniform(*p, n)
    return conservative(r, u, P, gamma).T.copy()


def random_smooth_field(rng, mesh: CartMesh, xi, amp=0.3, gamma=GAMMA, modes=3):
    """A smooth random admissible field: a sum of a few low Fourier modes in rho, u, v, P."""
    X = node_coords(mesh, xi)
    L = [mesh.hi[k] - mesh.lo[k] for k in range(mesh.dim)]

    def field_(base, a):
        f = np.full(X[0].shape, base, dtype=np.float64)
        for _ in range(modes):
            ph = rng.uniform(0, 2 * math.pi)
            arg = ph
            for k in range(mesh.dim):
                arg = arg + 2 * math.pi * rng.integers(1, 4) * (X[k] - mesh.lo[k]) / L[k]
            f = f + a * rng.uniform(-1, 1) * np.sin(arg)
        return f
    rho = field_(1.0, amp / modes)
    u = [field_(0.0, 0.5) for _ in range(mesh.dim)]
    P = field_(1.0, amp / modes)
    return np.ascontiguousarray(conservative(rho, u, P, gamma))


def random_discontinuous_field(rng, mesh: CartMesh, xi, gamma=GAMMA, jump=0.5):
    """Smooth field plus random per-element jumps and node noise: exercises the limiter."""
    w = random_smooth_field(rng, mesh, xi, gamma=gamma)
    E, ns = w.shape[1], w.shape[2]
    rho = w[0] * (1 + jump * rng.uniform(-0.5, 0.5, (E, 1))) * (1 + 0.2 * rng.uniform(-1, 1, (E, ns)))
    vel = [w[1 + k] / w[0] + 0.3 * rng.uniform(-1, 1, (E, ns)) for k in range(mesh.dim)]
    ke_old = 0.5 * sum((w[1 + k] / w[0]) ** 2 for k in range(mesh.dim)) * w[0]
    P = (gamma - 1) * (w[-1] - ke_old) * (1 + jump * rng.uniform(-0.5, 0.5, (E, 1)))
    P = P * (1 + 0.2 * rng.uniform(-1, 1, (E, ns)))
    return np.ascontiguousarray(conservative(rho, vel, P, gamma))


def four_quadrant_batch(seed, n_problems, n_range=(16, 128), p_range=(1, 4)):
    """Independent four-quadrant Riemann problems: per problem n ~ U{n_range} (n x n elements,
    rounded to even), p ~ U{p_range}, quadrant states from four_quadrant_states.  Returns a list
    of (p, mesh, ic) with Dirichlet boundary states per quadrant."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_problems):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        n += n % 2
        p = int(rng.integers(p_range[0], p_range[1] + 1))
        states = four_quadrant_states(rng)
        mesh, ic = four_quadrant(n, states)
        out.append((p, mesh, ic))
    return out


def batch_state(problems, nodes_of_p, state_offsets):
    """Concatenated initial state of a batch: problem i at state_offsets[i], layout [4][E_i][Ns_i];
    nodes_of_p(p) gives the reference nodes of order p."""
    w = np.zeros(int(state_offsets[-1]))
    for i, (p, mesh, ic) in enumerate(problems):
        a, b = int(state_offsets[i]), int(state_offsets[i + 1])
        w[a:b] = nodal_field(mesh, nodes_of_p(p), ic).ravel()
    return w


class TriMeshData:
    """An affine triangle mesh: xy[E][3][2] vertices (counterclockwise), nbr[E][3] (element across
    edge f, from vertex f to vertex f+1; negative = boundary id -(nbr+1)), nbr_edge[E][3] (the
    neighbour's matched edge), bc[n_bc][4]."""

    def __init__(self, xy, nbr, nbr_edge, bc, xy6=None):
        self.xy, self.nbr, self.nbr_edge, self.bc = xy, nbr, nbr_edge, bc
        self.xy6 = xy6   # curved elements: [E][6][2], the corners then the edges' mid-parameter points
        self.n_elem = nbr.shape[0]


def tri_mesh_2d(nx, ny, x0, x1, y0, y1, jitter=0.0, seed=0, periodic=(True, True)):
    """Unstructured-looking triangles on [x0,x1] x [y0,y1]: an nx x ny grid whose vertices are moved
    by up to jitter cell widths (seeded; the same move for periodic images), each cell cut into a
    lower-left (v00, v10, v01) and an upper-right (v10, v11, v01) triangle.  Element coordinates
    are unwrapped across periodic boundaries.  Non-periodic sides get boundary ids 0 (x) and 1 (y)."""
    rng = np.random.default_rng(seed)
    hx, hy = (x1 - x0) / nx, (y1 - y0) / ny
    mx, my = nx + 1, ny + 1
    jit = rng.uniform(-jitter, jitter, (mx, my, 2))
    if periodic[0]:
        jit[nx, :, :] = jit[0, :, :]
    else:
        jit[0, :, 0] = 0.0
        jit[nx, :, 0] = 0.0
    if periodic[1]:
        jit[:, ny, :] = jit[:, 0, :]
    else:
        jit[:, 0, 1] = 0.0
        jit[:, ny, 1] = 0.0

    def vert(i, j):
        return np.array([x0 + (i + jit[i, j, 0]) * hx, y0 + (j + jit[i, j, 1]) * hy])

    E = 2 * nx * ny
    xy = np.zeros((E, 3, 2))
    nbr = np.zeros((E, 3), np.int32)
    nbr_edge = np.zeros((E, 3), np.int32)

    def tid(i, j, t):
        return 2 * (j * nx + i) + t

    for j in range(ny):
        for i in range(nx):
            a, b = tid(i, j, 0), tid(i, j, 1)
            xy[a] = [vert(i, j), vert(i + 1, j), vert(i, j + 1)]
            xy[b] = [vert(i + 1, j), vert(i + 1, j + 1), vert(i, j + 1)]
            # lower-left: edge 0 bottom, 1 diagonal, 2 left; upper-right: 0 right, 1 top, 2 diagonal
            nbr[a, 1], nbr_edge[a, 1] = b, 2
            nbr[b, 2], nbr_edge[b, 2] = a, 1
            if j > 0 or periodic[1]:
                nbr[a, 0], nbr_edge[a, 0] = tid(i, (j - 1) % ny, 1), 1
            else:
                nbr[a, 0], nbr_edge[a, 0] = -2, 0
            if i > 0 or periodic[0]:
                nbr[a, 2], nbr_edge[a, 2] = tid((i - 1) % nx, j, 1), 0
            else:
                nbr[a, 2], nbr_edge[a, 2] = -1, 0
            if i < nx - 1 or periodic[0]:
                nbr[b, 0], nbr_edge[b, 0] = tid((i + 1) % nx, j, 0), 2
            else:
                nbr[b, 0], nbr_edge[b, 0] = -1, 0
            if j < ny - 1 or periodic[1]:
                nbr[b, 1], nbr_edge[b, 1] = tid(i, (j + 1) % ny, 0), 0
            else:
                nbr[b, 1], nbr_edge[b, 1] = -2, 0
    bc = np.array([[1.0, 0.0, 0.0, 2.5], [1.0, 0.0, 0.0, 2.5]])
    return TriMeshData(xy, nbr, nbr_edge, bc)


def tri_curved_mesh(nx, ny, x0, x1, y0, y1, jitter=0.0, bump=0.15, seed=0, periodic=(True, True)):
    """tri_mesh_2d with curved (quadratic) elements: each edge's mid-parameter point is its
    midpoint moved by bump cell widths times a smooth field periodic over the domain, evaluated at
    the midpoint itself, so that the two elements of an edge (and periodic images) agree."""
    m = tri_mesh_2d(nx, ny, x0, x1, y0, y1, jitter=jitter, seed=seed, periodic=periodic)
    hx, hy = (x1 - x0) / nx, (y1 - y0) / ny
    Lx, Ly = x1 - x0, y1 - y0
    xy6 = np.zeros((m.n_elem, 6, 2))
    xy6[:, :3] = m.xy
    for f in range(3):
        mid = 0.5 * (m.xy[:, f] + m.xy[:, (f + 1) % 3])
        px, py = 2 * np.pi * (mid[:, 0] - x0) / Lx, 2 * np.pi * (mid[:, 1] - y0) / Ly
        xy6[:, 3 + f, 0] = mid[:, 0] + bump * hx * np.sin(py) * np.cos(px + 0.3)
        xy6[:, 3 + f, 1] = mid[:, 1] + bump * hy * np.sin(px) * np.cos(py + 0.7)
    m.xy6 = xy6
    return m


def tri_positions(mesh, rs):
    """Physical positions x[E][n], y[E][n] of reference points rs[n][2] on every triangle: the
    affine map of the corners, or the quadratic map of xy6 on curved meshes."""
    r, s = rs[None, :, 0], rs[None, :, 1]
    if getattr(mesh, "xy6", None) is not None:
        l1, l2, l3 = 1 - r - s, r, s
        N = [l1 * (2 * l1 - 1), l2 * (2 * l2 - 1), l3 * (2 * l3 - 1), 4 * l1 * l2, 4 * l2 * l3, 4 * l3 * l1]
        x = sum(N[k] * mesh.xy6[:, k, 0][:, None] for k in range(6))
        y = sum(N[k] * mesh.xy6[:, k, 1][:, None] for k in range(6))
        return x, y
    X0 = mesh.xy[:, 0, :]
    J1 = mesh.xy[:, 1, :] - X0
    J2 = mesh.xy[:, 2, :] - X0
    x = X0[:, None, 0] + r * J1[:, None, 0] + s * J2[:, None, 0]
    y = X0[:, None, 1] + r * J1[:, None, 1] + s * J2[:, None, 1]
    return x, y


def tri_nodal_field(mesh, rs, ic):
    """Initial state at the solution points of every triangle, w[E][ns][4]; rs[ns][2] reference
    points on (0,0), (1,0), (0,1), ic(x, y) -> (4, ...) conservative state."""
    x, y = tri_positions(mesh, rs)
    q = np.asarray(ic(x, y), dtype=np.float64)          # [4][E][ns]
    return np.ascontiguousarray(np.moveaxis(q, 0, -1))  # [E][ns][4]


def tri_blast(x, y, gamma=1.4):
    """Smoothed circular blast on [0,1]^2 with a weak shear: density 1 / 0.125 and pressure 1 / 0.1
    inside / outside radius 0.25 about (0.5, 0.5), joined by a tanh front of width 0.01 (about 2.5
    cells of a 256^2 mesh), velocity (0.2 sin 2 pi y, -0.2 sin 2 pi x).  Conservative state
    (4, ...)."""
    s = 0.5 * (1 - np.tanh((np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2) - 0.25) / 0.01))
    rho = 0.125 + 0.875 * s
    P = 0.1 + 0.9 * s
    u = 0.2 * np.sin(2 * np.pi * y)
    v = -0.2 * np.sin(2 * np.pi * x)
    return np.stack([rho, rho * u, rho * v, P / (gamma - 1) + 0.5 * rho * (u * u + v * v)])
