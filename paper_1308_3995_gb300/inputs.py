"""Seeded synthetic inputs: periodic jittered triangle meshes, degree maps and
coefficient vectors of a Newton iterate.

This module is data only.  It holds none of the HDG method's arithmetic (no
basis, quadrature, flux, Jacobian or condensation): both the CUDA path and
the CPU oracle receive exactly the arrays built here.  The flow conditions
follow the paper's test cases (arXiv:1308.3995, Sec. 5: gamma = 1.4, Mach
0.5/0.8/1.4, Re = 5000, Pr = 0.72; degrees p = 1..4); the meshes replace the
NACA0012 meshes, which are not available, by periodic unit-square grids.

Recipe (all random numbers from ``numpy.random.default_rng(seed)``):
  * mesh: nx x ny cells of the unit square, periodic; cell (i, j) split along
    its (i,j)-(i+1,j+1) diagonal into (a,b,c) and (a,c,d) (counter-clockwise);
    each topological vertex moved by U(-j hx, j hx) x U(-j hy, j hy); element
    vertex coordinates carry the periodic image (+1) where a cell wraps;
  * state: the analytic primitive field (rho, u, v, p) of the case is turned
    into conserved variables (rho, rho u, rho v, p/(gamma-1) + rho|v|^2/2);
    mode 0 of each element's coefficients is the field at the centroid
    divided by sqrt(2) (sqrt(2) is the value of the constant mode of an
    orthonormal basis on a reference triangle of area 1/2), modes m >= 1 are
    1e-3 * scale_f * N(0,1) / (m+1); Navier-Stokes gradient coefficients are
    5e-2 * scale_f * N(0,1) for mode 0 and 1e-3 * scale_f * N(0,1)/(m+1)
    otherwise; scale_f = |w_inf,f| + 0.1;
  * trace: mode 0 of every face is the field at the face midpoint, modes
    k >= 1 are 1e-3 * scale_f * N(0,1) / (k+1);
  * trace update for the reconstruction: 1e-3 * N(0,1) per entry.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SQRT2 = math.sqrt(2.0)


# --------------------------------------------------------------------------- meshes
@dataclass
class MeshData:
    nx: int
    ny: int
    elem_xy: np.ndarray      # [n_elem, 3, 2] float64, CCW, periodic images resolved
    elem_vid: np.ndarray     # [n_elem, 3] int32 topological vertex ids
    vert_xy: np.ndarray      # [n_vert, 2] jittered positions in [0,1)^2 (mod 1)
    elem_bc: np.ndarray | None = None   # [n_elem, 3] int8 boundary kind of local face l (0 interior)

    @property
    def n_elem(self) -> int:
        return int(self.elem_vid.shape[0])

    @property
    def h(self) -> float:
        return 1.0 / max(self.nx, self.ny)


def periodic_mesh(nx: int, ny: int, jitter: float, seed: int) -> MeshData:
    if nx < 3 or ny < 3:
        raise ValueError("periodic grids need at least 3 cells per direction")
    rng = np.random.default_rng(seed)
    hx, hy = 1.0 / nx, 1.0 / ny
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")  # [ny, nx]
    jx = rng.uniform(-jitter * hx, jitter * hx, size=(ny, nx)) if jitter > 0 else np.zeros((ny, nx))
    jy = rng.uniform(-jitter * hy, jitter * hy, size=(ny, nx)) if jitter > 0 else np.zeros((ny, nx))
    X = ii * hx + jx
    Y = jj * hy + jy
    vid = (jj * nx + ii).astype(np.int64)

    def corner(di, dj):
        i2 = (ii + di) % nx
        j2 = (jj + dj) % ny
        x = X[j2, i2] + (ii + di >= nx)
        y = Y[j2, i2] + (jj + dj >= ny)
        return np.stack([x, y], -1), vid[j2, i2]

    a, va = corner(0, 0)
    b, vb = corner(1, 0)
    c, vc = corner(1, 1)
    d, vd = corner(0, 1)
    t1 = np.stack([a, b, c], -2)          # [ny, nx, 3, 2]
    t2 = np.stack([a, c, d], -2)
    v1 = np.stack([va, vb, vc], -1)
    v2 = np.stack([va, vc, vd], -1)
    elem_xy = np.stack([t1, t2], 2).reshape(-1, 3, 2)
    elem_vid = np.stack([v1, v2], 2).reshape(-1, 3).astype(np.int32)
    e = elem_xy
    det = (e[:, 1, 0] - e[:, 0, 0]) * (e[:, 2, 1] - e[:, 0, 1]) - (e[:, 2, 0] - e[:, 0, 0]) * (e[:, 1, 1] - e[:, 0, 1])
    if not np.all(det > 0):
        raise ValueError("jitter produced a non-positive element")
    vert_xy = np.stack([X.reshape(-1), Y.reshape(-1)], -1)
    return MeshData(nx, ny, np.ascontiguousarray(elem_xy), elem_vid, vert_xy)


BC_SLIP_WALL, BC_FAR_FIELD, BC_NO_SLIP_WALL = 1, 2, 3


def channel_mesh(nx: int, ny: int, jitter: float, seed: int, bottom: int = BC_SLIP_WALL,
                 top: int = BC_FAR_FIELD) -> MeshData:
    """Unit square, periodic in x, bounded in y: a slip wall along y = 0 and a far-field boundary
    along y = 1 (boundary kinds as given).  Same cell split as the periodic mesh; interior vertex rows
    jittered in x and y, the two boundary rows in x only."""
    if nx < 3 or ny < 2:
        raise ValueError("channel grids need nx >= 3 and ny >= 2")
    rng = np.random.default_rng(seed)
    hx, hy = 1.0 / nx, 1.0 / ny
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny + 1), indexing="xy")  # [ny+1, nx]
    jx = rng.uniform(-jitter * hx, jitter * hx, size=(ny + 1, nx)) if jitter > 0 else np.zeros((ny + 1, nx))
    jy = rng.uniform(-jitter * hy, jitter * hy, size=(ny + 1, nx)) if jitter > 0 else np.zeros((ny + 1, nx))
    jy[0, :] = 0.0
    jy[ny, :] = 0.0
    X = ii * hx + jx
    Y = jj * hy + jy
    vid = (jj * nx + ii).astype(np.int64)
    ic, jc = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")      # cells [ny, nx]

    def corner(di, dj):
        i2 = (ic + di) % nx
        j2 = jc + dj
        x = X[j2, i2] + (ic + di >= nx)
        return np.stack([x, Y[j2, i2]], -1), vid[j2, i2]

    a, va = corner(0, 0)
    b, vb = corner(1, 0)
    c, vc = corner(1, 1)
    d, vd = corner(0, 1)
    t1 = np.stack([a, b, c], -2)
    t2 = np.stack([a, c, d], -2)
    v1 = np.stack([va, vb, vc], -1)
    v2 = np.stack([va, vc, vd], -1)
    elem_xy = np.stack([t1, t2], 2).reshape(-1, 3, 2)
    elem_vid = np.stack([v1, v2], 2).reshape(-1, 3).astype(np.int32)
    bc = np.zeros((ny, nx, 2, 3), np.int8)
    bc[0, :, 0, 0] = bottom        # (a, b) of the lower triangle on y = 0
    bc[ny - 1, :, 1, 1] = top      # (c, d) of the upper triangle on y = 1
    e = elem_xy
    det = (e[:, 1, 0] - e[:, 0, 0]) * (e[:, 2, 1] - e[:, 0, 1]) - (e[:, 2, 0] - e[:, 0, 0]) * (e[:, 1, 1] - e[:, 0, 1])
    if not np.all(det > 0):
        raise ValueError("jitter produced a non-positive element")
    vert_xy = np.stack([X.reshape(-1), Y.reshape(-1)], -1)
    return MeshData(nx, ny, np.ascontiguousarray(elem_xy), elem_vid, vert_xy, bc.reshape(-1, 3))


def box_mesh(nx: int, ny: int, jitter: float, seed: int, kind: int = BC_FAR_FIELD) -> MeshData:
    """Unit square bounded on all four sides by boundary faces of one kind (far field by default).
    Same cell split; interior vertices jittered in x and y, boundary vertices along their side only,
    corners fixed."""
    if nx < 2 or ny < 2:
        raise ValueError("box grids need at least 2 cells per direction")
    rng = np.random.default_rng(seed)
    hx, hy = 1.0 / nx, 1.0 / ny
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")  # [ny+1, nx+1]
    jx = rng.uniform(-jitter * hx, jitter * hx, size=ii.shape) if jitter > 0 else np.zeros(ii.shape)
    jy = rng.uniform(-jitter * hy, jitter * hy, size=ii.shape) if jitter > 0 else np.zeros(ii.shape)
    jx[:, 0] = 0.0; jx[:, nx] = 0.0
    jy[0, :] = 0.0; jy[ny, :] = 0.0
    X = ii * hx + jx
    Y = jj * hy + jy
    vid = (jj * (nx + 1) + ii).astype(np.int64)
    ic, jc = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")

    def corner(di, dj):
        return np.stack([X[jc + dj, ic + di], Y[jc + dj, ic + di]], -1), vid[jc + dj, ic + di]

    a, va = corner(0, 0)
    b, vb = corner(1, 0)
    c, vc = corner(1, 1)
    d, vd = corner(0, 1)
    elem_xy = np.stack([np.stack([a, b, c], -2), np.stack([a, c, d], -2)], 2).reshape(-1, 3, 2)
    elem_vid = np.stack([np.stack([va, vb, vc], -1), np.stack([va, vc, vd], -1)], 2).reshape(-1, 3).astype(np.int32)
    bc = np.zeros((ny, nx, 2, 3), np.int8)
    bc[0, :, 0, 0] = kind          # (a, b) on y = 0
    bc[:, nx - 1, 0, 1] = kind     # (b, c) on x = 1
    bc[ny - 1, :, 1, 1] = kind     # (c, d) on y = 1
    bc[:, 0, 1, 2] = kind          # (d, a) on x = 0
    e = elem_xy
    det = (e[:, 1, 0] - e[:, 0, 0]) * (e[:, 2, 1] - e[:, 0, 1]) - (e[:, 2, 0] - e[:, 0, 0]) * (e[:, 1, 1] - e[:, 0, 1])
    if not np.all(det > 0):
        raise ValueError("jitter produced a non-positive element")
    vert_xy = np.stack([X.reshape(-1), Y.reshape(-1)], -1)
    return MeshData(nx, ny, np.ascontiguousarray(elem_xy), elem_vid, vert_xy, bc.reshape(-1, 3))


def degree_map(n_elem: int, seed: int, p: int | None = None, probs=None) -> np.ndarray:
    """Uniform degree p, or i.i.d. degrees 1..4 with the given probabilities."""
    if p is not None:
        return np.full(n_elem, p, dtype=np.int8)
    rng = np.random.default_rng(seed)
    return rng.choice(np.arange(1, 5), size=n_elem, p=probs).astype(np.int8)


# --------------------------------------------------------------------------- flow fields
def free_stream(mach: float, aoa_deg: float, gamma: float = 1.4):
    a = math.radians(aoa_deg)
    return 1.0, mach * math.cos(a), mach * math.sin(a), 1.0 / gamma


def conserved(rho, u, v, p, gamma=1.4):
    rho, u, v, p = (np.asarray(t, dtype=np.float64) for t in (rho, u, v, p))
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)], -1)


class Field:
    """Analytic periodic primitive field on [0,1)^2."""

    def __init__(self, kind: str, mach: float, aoa: float, seed: int, gamma: float = 1.4, h: float = 1 / 64,
                 kvec=None):
        self.kind, self.gamma = kind, gamma
        self.rho0, self.u0, self.v0, self.p0 = free_stream(mach, aoa, gamma)
        rng = np.random.default_rng(seed)
        if kind == "bump":
            self.center = rng.uniform(0.0, 1.0, size=2)
            self.amp, self.sigma = 0.05, 0.1
        elif kind == "fourier":
            ks = [(kx, ky) for kx in range(-2, 3) for ky in range(-2, 3) if (kx, ky) != (0, 0)]
            self.k = np.array(ks, dtype=np.float64)
            damp = 0.01 / (1.0 + (self.k ** 2).sum(1))
            self.amp = damp[:, None] * rng.standard_normal((len(ks), 4))
            self.phase = rng.uniform(0.0, 2 * math.pi, size=(len(ks), 4))
        elif kind == "shock":
            choices = [(1, 0), (2, 1), (3, 1), (1, 1), (2, -1), (3, -1)]
            pick = choices[int(rng.integers(len(choices)))]
            self.kvec = np.array(kvec if kvec is not None else pick, dtype=np.float64)
            kn = np.linalg.norm(self.kvec)
            nrm = self.kvec / kn
            un1 = self.u0 * nrm[0] + self.v0 * nrm[1]
            ut1 = -self.u0 * nrm[1] + self.v0 * nrm[0]
            c1 = math.sqrt(gamma * self.p0 / self.rho0)
            M = un1 / c1
            if M <= 1.0:
                raise ValueError("shock band needs a supersonic normal Mach number")
            g = gamma
            r = (g + 1) * M * M / ((g - 1) * M * M + 2)          # normal-shock density ratio
            self.rho1 = self.rho0 * r
            self.p1 = self.p0 * (1 + 2 * g / (g + 1) * (M * M - 1))
            un2 = un1 / r
            self.u1 = un2 * nrm[0] - ut1 * nrm[1]
            self.v1 = un2 * nrm[1] + ut1 * nrm[0]
            self.width = 2.0 * h * kn                             # tanh width in phase units
        elif kind != "uniform":
            raise ValueError(kind)

    def primitive(self, x, y):
        x = np.asarray(x, np.float64); y = np.asarray(y, np.float64)
        rho = np.full_like(x, self.rho0); u = np.full_like(x, self.u0)
        v = np.full_like(x, self.v0); p = np.full_like(x, self.p0)
        if self.kind == "bump":
            dx = (x - self.center[0] + 0.5) % 1.0 - 0.5
            dy = (y - self.center[1] + 0.5) % 1.0 - 0.5
            rho = rho + self.amp * np.exp(-(dx * dx + dy * dy) / (2 * self.sigma ** 2))
        elif self.kind == "fourier":
            arg = 2 * math.pi * (np.multiply.outer(x, self.k[:, 0]) + np.multiply.outer(y, self.k[:, 1]))
            pert = [(self.amp[:, c] * np.cos(arg + self.phase[:, c])).sum(-1) for c in range(4)]
            rho, u, v, p = rho + pert[0], u + pert[1], v + pert[2], p + pert[3]
        elif self.kind == "shock":
            th = (self.kvec[0] * x + self.kvec[1] * y) % 1.0
            chi = 0.5 * (np.tanh((th - 0.25) / self.width) - np.tanh((th - 0.75) / self.width))
            rho = (1 - chi) * self.rho0 + chi * self.rho1
            u = (1 - chi) * self.u0 + chi * self.u1
            v = (1 - chi) * self.v0 + chi * self.v1
            p = (1 - chi) * self.p0 + chi * self.p1
        return rho, u, v, p

    def conserved(self, x, y):
        return conserved(*self.primitive(x, y), gamma=self.gamma)

    @property
    def w_inf(self):
        return conserved(self.rho0, self.u0, self.v0, self.p0, self.gamma)


def _n_basis(p):
    return (p + 1) * (p + 2) // 2


def element_coeffs(mesh: MeshData, elem_p: np.ndarray, fld: Field, nfield: int, seed: int) -> np.ndarray:
    """Coefficient vector U (elements in order; per element [fields][modes],
    Navier-Stokes fields ordered q_x(4), q_y(4), w(4))."""
    rng = np.random.default_rng(seed)
    cen = mesh.elem_xy.mean(1) % 1.0
    wc = fld.conserved(cen[:, 0], cen[:, 1])                  # [n_elem, 4]
    scale = np.abs(fld.w_inf) + 0.1
    n_of = np.array([nfield * _n_basis(int(p)) for p in range(5)], dtype=np.int64)[elem_p.astype(np.int64)]
    off = np.concatenate([[0], np.cumsum(n_of)])
    U = np.zeros(int(off[-1]))
    for p in range(1, 5):
        idx = np.nonzero(elem_p == p)[0]
        if idx.size == 0:
            continue
        nb = _n_basis(p)
        m = np.arange(nb)
        w = 1e-3 * scale[None, :, None] * rng.standard_normal((idx.size, 4, nb)) / (m + 1)[None, None, :]
        w[:, :, 0] = wc[idx] / SQRT2
        blocks = [w]
        if nfield == 12:
            q = 1e-3 * scale[None, None, :, None] * rng.standard_normal((idx.size, 2, 4, nb)) / (m + 1)
            q[:, :, :, 0] = 5e-2 * scale[None, None, :] * rng.standard_normal((idx.size, 2, 4))
            blocks = [q.reshape(idx.size, 8, nb), w]
        vals = np.concatenate(blocks, 1).reshape(idx.size, -1)
        U[(off[idx][:, None] + np.arange(vals.shape[1])[None, :]).ravel()] = vals.ravel()
    return U


def trace_coeffs(mesh: MeshData, face_vid: np.ndarray, face_p: np.ndarray, fld: Field, seed: int) -> np.ndarray:
    """Trace vector Lambda (faces in the given order; per face [fields][modes])."""
    rng = np.random.default_rng(seed)
    a = mesh.vert_xy[face_vid[:, 0]]
    b = mesh.vert_xy[face_vid[:, 1]]
    d = (b - a + 0.5) % 1.0 - 0.5                              # minimal periodic image
    mid = (a + 0.5 * d) % 1.0
    wm = fld.conserved(mid[:, 0], mid[:, 1])
    scale = np.abs(fld.w_inf) + 0.1
    nk = face_p.astype(np.int64) + 1
    off = np.concatenate([[0], np.cumsum(4 * nk)])
    out = np.zeros(int(off[-1]))
    noise = rng.standard_normal(int(off[-1]))
    for k in np.unique(nk):
        idx = np.nonzero(nk == k)[0]
        kk = np.arange(k)
        c = 1e-3 * scale[None, :, None] * noise[(off[idx][:, None] + np.arange(4 * k)[None, :])].reshape(-1, 4, k) \
            / (kk + 1)[None, None, :]
        c[:, :, 0] = wm[idx]
        out[(off[idx][:, None] + np.arange(4 * k)[None, :]).ravel()] = c.ravel()
    return out


def trace_update(lam_len: int, seed: int) -> np.ndarray:
    return 1e-3 * np.random.default_rng(seed).standard_normal(lam_len)


# --------------------------------------------------------------------------- named workloads
@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    jitter: float
    model: int                 # 0 Euler, 1 NS mixed form
    p: int | None              # uniform degree, or None for the mix
    probs: tuple | None
    field: str
    mach: float
    aoa: float
    reynolds: float = 5000.0
    prandtl: float = 0.72
    seed: int = 1234
    extra: dict = field(default_factory=dict)
    # "channel": slip wall at y = 0, far field at y = 1; "box": far field all round;
    # "wall_channel": no-slip adiabatic walls at y = 0 and y = 1 (Navier-Stokes);
    # "wall_far_channel": a no-slip adiabatic wall at y = 0, far field at y = 1 (Navier-Stokes)
    domain: str = "periodic"

    @property
    def n_elem(self) -> int:
        return 2 * self.nx * self.ny

    @property
    def alpha(self) -> float:
        # free-stream maximal wave speed |v_inf| + c_inf with c_inf = 1
        return self.mach + 1.0


WORKLOADS = {
    # 256 triangles, Euler p=1, Mach 0.5 / 2 deg + Gaussian density bump
    "euler_p1_256": Workload("euler_p1_256", 8, 16, 0.0, 0, 1, None, "bump", 0.5, 2.0, seed=11),
    # 16,384 jittered triangles, Euler p=3, Mach 0.8 / 1.25 deg + Fourier modes
    "euler_p3_16k": Workload("euler_p3_16k", 64, 128, 0.2, 0, 3, None, "fourier", 0.8, 1.25, seed=22),
    # 65,536 jittered triangles, NS mixed form, p in {1,2,3,4} at 40/30/20/10 %
    "ns_mixp_65k": Workload("ns_mixp_65k", 128, 256, 0.2, 1, None, (0.4, 0.3, 0.2, 0.1), "fourier", 0.5, 1.0,
                            seed=33),
    # 262,144 jittered triangles, Euler p=3, Mach 1.5 oblique shock band
    "euler_p3_262k_shock": Workload("euler_p3_262k_shock", 256, 512, 0.2, 0, 3, None, "shock", 1.5, 0.0, seed=44),
    # bounded domain: 8,192 jittered triangles between a slip wall (y = 0) and a far field (y = 1),
    # Euler p=2, Mach 0.5 free stream along the wall + Gaussian density bump
    "euler_channel_8k": Workload("euler_channel_8k", 64, 64, 0.2, 0, 2, None, "bump", 0.5, 0.0, seed=55,
                                 domain="channel"),
    # far field on all four sides of the unit square: 8,192 jittered triangles, Euler p=2, Mach 0.5 at
    # 10 degrees + Gaussian density bump, which the steady solve washes out to the free stream
    "euler_box_8k": Workload("euler_box_8k", 64, 64, 0.2, 0, 2, None, "bump", 0.5, 10.0, seed=66, domain="box"),
    # Navier-Stokes between two no-slip adiabatic walls (y = 0, y = 1), periodic in x: 8,192 jittered
    # triangles, p in {1,2,3,4} at 40/30/20/10 %, Mach 0.5, Re 5000, Fourier modes on the free stream
    "ns_wall_channel_8k": Workload("ns_wall_channel_8k", 64, 64, 0.2, 1, None, (0.4, 0.3, 0.2, 0.1), "fourier",
                                   0.5, 0.0, seed=77, domain="wall_channel"),
    # Navier-Stokes with far field on all four sides (Mach 0.5 at 10 degrees + density bump)
    "ns_box_8k": Workload("ns_box_8k", 64, 64, 0.2, 1, 2, None, "bump", 0.5, 10.0, seed=88, domain="box"),
}


def small_variant(w: Workload, nx: int, ny: int, **kw) -> Workload:
    d = dict(w.__dict__)
    d.update(nx=nx, ny=ny, name=f"{w.name}@{nx}x{ny}")
    d.update(kw)
    return Workload(**d)


@dataclass
class Case:
    wl: Workload
    mesh: MeshData
    elem_p: np.ndarray
    fld: Field

    @property
    def nfield(self):
        return 12 if self.wl.model == 1 else 4


def make_case(wl: Workload) -> Case:
    if wl.domain == "channel":
        mesh = channel_mesh(wl.nx, wl.ny, wl.jitter, wl.seed)
    elif wl.domain == "wall_channel":
        mesh = channel_mesh(wl.nx, wl.ny, wl.jitter, wl.seed, bottom=BC_NO_SLIP_WALL, top=BC_NO_SLIP_WALL)
    elif wl.domain == "wall_far_channel":   # a boundary layer: no-slip wall below, far field above
        mesh = channel_mesh(wl.nx, wl.ny, wl.jitter, wl.seed, bottom=BC_NO_SLIP_WALL, top=BC_FAR_FIELD)
    elif wl.domain == "box":
        mesh = box_mesh(wl.nx, wl.ny, wl.jitter, wl.seed)
    else:
        mesh = periodic_mesh(wl.nx, wl.ny, wl.jitter, wl.seed)
    ep = degree_map(mesh.n_elem, wl.seed + 1, p=wl.p, probs=wl.probs)
    fld = Field(wl.field, wl.mach, wl.aoa, wl.seed + 2, h=mesh.h, kvec=wl.extra.get("kvec"))
    return Case(wl, mesh, ep, fld)


def case_state(case: Case, face_vid: np.ndarray, face_p: np.ndarray):
    """U, Lambda and a trace update for a case, given the face list (lo, hi
    vertex ids) and face degrees of its mesh."""
    U = element_coeffs(case.mesh, case.elem_p, case.fld, case.nfield, case.wl.seed + 3)
    Lam = trace_coeffs(case.mesh, face_vid, face_p, case.fld, case.wl.seed + 4)
    dLam = trace_update(Lam.size, case.wl.seed + 5)
    return U, Lam, dLam
