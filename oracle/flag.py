"""Spring-network flag (Sec. II.B, structural model; Sec. II.A, flag problem).

The flag is a square sheet hinged at its leading edge (LE) with its other
edges free, meshed by a structured lattice of ns x nt vertices. Each lattice cell is
split into two right triangles in two ways (along either diagonal); both
triangulations carry bending hinges with weight 1/2 each, because a single
split direction couples bending to twist and lowers the first bending
frequency by about a third. Masses sit on the vertices; in-plane springs on every
lattice edge and diagonal make the sheet essentially inextensible, and
out-of-plane (dihedral) springs on every interior edge carry the bending
stiffness.

Energies (the paper gives no spring constants; readings stated here):
    E_s = k_s / 2 * sum_springs (|x_a - x_b| - l0)^2      (k_s = 1000)
    E_b = sum_hinges k_e (1 - n_A . n_B)
Springs sit on every lattice edge and on both diagonals of every cell. n_A,
n_B are the unit normals of the two triangles (of one triangulation) sharing
a hinge edge e of rest length |e|; with cell area A = ds dt,
    k_e = (1/2) beta |e|^2 / A        on lattice edges,
    k_e = (1/2) 2 beta A / |e|^2      on diagonals.
For cylindrical bending of curvature kappa along either lattice axis one
lattice edge per cell turns by kappa times the cell side across it and the
diagonals stay flat; for a twist kappa_st only the diagonals turn. The
small-deflection energy density is therefore
(beta / 2)(kappa_ss^2 + kappa_tt^2 + 2 kappa_st^2), the Kirchhoff plate with
Poisson ratio 0, where beta = B / (rho_f U^2 L^3) is the paper's bending
coefficient.

Forces are minus the gradient of E_s + E_b, taken by automatic
differentiation of the energy (PyTorch CPU, FP64). LE vertices are held fixed
(the hinge transmits no moment because no bending spring crosses the LE).

Time integration: velocity Verlet with n_sub equal sub-steps per fluid step,
n_sub = ceil(dt * omega_max / 1.8): velocity Verlet is stable for
dt_s * omega < 2, and omega_max bounds the linearised stiffness-over-mass
spectrum from above by Gershgorin's theorem, so dt_s * omega <= 1.8:
    omega_max^2 = max_v (2 k_s n_springs(v) + 8 sum_{hinges at v} k_e / l_min^2) / m_v
over free vertices. The fluid force is held constant over the sub-steps.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def vid(a, b, nt):
    """Vertex index of lattice point (a, b) (a along the chord from the hinged
    leading edge, b along the span), nt vertices per spanwise row (Sec. II.A)."""
    return a * nt + b


class FlagMesh:
    """Lattice, springs, hinges, lumped areas and masses of the flag."""

    def __init__(self, ns, nt, length, span, rho, k_s, k_b):
        self.ns, self.nt = ns, nt
        self.ds = length / (ns - 1)
        self.dt = span / (nt - 1)
        self.k_s, self.k_b, self.rho = k_s, k_b, rho
        nv = ns * nt
        self.nv = nv
        # two overlaid triangulations, each with triangles CCW in the (s, t)
        # parameter plane: A splits every cell along (a,b)-(a+1,b+1), B along
        # (a+1,b)-(a,b+1). Either one alone couples bending to twist (with
        # opposite signs); the bending energy averages the two.
        tris, kinds = [], []
        for split in (0, 1):
            for a in range(ns - 1):
                for b in range(nt - 1):
                    v00, v10 = vid(a, b, nt), vid(a + 1, b, nt)
                    v01, v11 = vid(a, b + 1, nt), vid(a + 1, b + 1, nt)
                    if split == 0:
                        tris += [(v00, v10, v11), (v00, v11, v01)]
                    else:
                        tris += [(v00, v10, v01), (v10, v11, v01)]
                    kinds += [split, split]
        self.tris = np.array(tris, dtype=np.int64)
        # springs: lattice edges along s and t, plus both cell diagonals
        springs = []
        for a in range(ns):
            for b in range(nt):
                if a + 1 < ns:
                    springs.append((vid(a, b, nt), vid(a + 1, b, nt)))
                if b + 1 < nt:
                    springs.append((vid(a, b, nt), vid(a, b + 1, nt)))
        for a in range(ns - 1):
            for b in range(nt - 1):
                springs.append((vid(a, b, nt), vid(a + 1, b + 1, nt)))
                springs.append((vid(a + 1, b, nt), vid(a, b + 1, nt)))
        self.springs = np.array(springs, dtype=np.int64)
        # hinges: pairs of triangles of the same triangulation sharing an edge
        edge_tris = {}
        for t, tri in enumerate(self.tris):
            for e in range(3):
                p, q = tri[e], tri[(e + 1) % 3]
                key = (kinds[t], min(p, q), max(p, q))
                edge_tris.setdefault(key, []).append(t)
        hinges = [(ts[0], ts[1], key[1:]) for key, ts in edge_tris.items() if len(ts) == 2]
        self.hinge_tris = np.array([(h[0], h[1]) for h in hinges], dtype=np.int64)
        self.hinge_edges = np.array([h[2] for h in hinges], dtype=np.int64)
        # hinge stiffness (each triangulation carries weight 1/2): lattice
        # edges k = beta |e|^2 / A_cell, diagonals k = 2 beta A_cell / |e|^2,
        # which makes the small-deflection energy density
        # (beta / 2) (k_ss^2 + k_tt^2 + 2 k_st^2), an isotropic plate with
        # Poisson ratio 0
        st = np.array([[a * self.ds, b * self.dt] for a in range(ns) for b in range(nt)])
        e = st[self.hinge_edges[:, 1]] - st[self.hinge_edges[:, 0]]
        e2 = (e * e).sum(axis=1)
        cell = self.ds * self.dt
        diagonal = (np.abs(e[:, 0]) > 0) & (np.abs(e[:, 1]) > 0)
        self.k_hinge = 0.5 * np.where(diagonal, 2.0 * k_b * cell / e2, k_b * e2 / cell)
        # lumped areas: a quarter of each adjacent lattice cell
        area = np.zeros(nv)
        cell = self.ds * self.dt
        for a in range(ns - 1):
            for b in range(nt - 1):
                for (aa, bb) in ((a, b), (a + 1, b), (a, b + 1), (a + 1, b + 1)):
                    area[vid(aa, bb, nt)] += 0.25 * cell
        self.area = area
        self.mass = rho * area
        self.free = np.ones(nv, dtype=bool)
        self.free[[vid(0, b, nt) for b in range(nt)]] = False

    def initial_positions(self, x_le, yc, zc, span, pitch):
        """Straight flag at pitch angle theta0 about the spanwise (z) axis."""
        X = np.zeros((self.ns, self.nt, 3))
        s = np.arange(self.ns) * self.ds
        t = np.arange(self.nt) * self.dt
        X[:, :, 0] = (x_le + s * math.cos(pitch))[:, None]
        X[:, :, 1] = (yc + s * math.sin(pitch))[:, None]
        X[:, :, 2] = (zc - 0.5 * span + t)[None, :]
        return X.reshape(-1, 3)

    def rest_lengths(self, X0):
        """Spring rest lengths l0 = |X_b - X_a| in the flat reference state X0
        (the stretching springs of Sec. II.A hold the sheet near inextensible)."""
        d = X0[self.springs[:, 1]] - X0[self.springs[:, 0]]
        return np.sqrt((d * d).sum(axis=1))

    def omega_max(self):
        """Gershgorin bound of the linearised stiffness-over-mass spectrum."""
        n_spr = np.bincount(self.springs.reshape(-1), minlength=self.nv)
        k_hinge_sum = np.zeros(self.nv)
        for (t0, t1), k in zip(self.hinge_tris, self.k_hinge):
            for v in set(self.tris[t0]) | set(self.tris[t1]):
                k_hinge_sum[v] += k
        lmin = min(self.ds, self.dt)
        w2 = (2.0 * self.k_s * n_spr + 8.0 * k_hinge_sum / lmin ** 2) / self.mass
        return math.sqrt(float(np.max(w2[self.free])))

    def substeps(self, dt):
        """Velocity-Verlet sub-steps per fluid step (Sec. II.B: the structure
        advances in smaller steps): ceil(dt omega_max / 1.8), so every mode
        runs at dt_s omega <= 1.8 below the stability limit 2."""
        return max(1, int(math.ceil(dt * self.omega_max() / 1.8)))


def energy(X, mesh, l0):
    """E_s + E_b for positions X (torch, (nv, 3), float64)."""
    sp = torch.as_tensor(mesh.springs)
    d = X[sp[:, 1]] - X[sp[:, 0]]
    length = torch.sqrt((d * d).sum(dim=1))
    e_s = 0.5 * mesh.k_s * ((length - torch.as_tensor(l0)) ** 2).sum()
    tr = torch.as_tensor(mesh.tris)
    n = torch.cross(X[tr[:, 1]] - X[tr[:, 0]], X[tr[:, 2]] - X[tr[:, 0]], dim=1)
    n = n / torch.sqrt((n * n).sum(dim=1, keepdim=True))
    ht = torch.as_tensor(mesh.hinge_tris)
    cos = (n[ht[:, 0]] * n[ht[:, 1]]).sum(dim=1)
    e_b = (torch.as_tensor(mesh.k_hinge) * (1.0 - cos)).sum()
    return e_s + e_b


def elastic_forces(X, mesh, l0):
    """-dE/dX at X (numpy (nv, 3)) by automatic differentiation."""
    Xt = torch.tensor(X, dtype=torch.float64, requires_grad=True)
    e = energy(Xt, mesh, l0)
    (g,) = torch.autograd.grad(e, Xt)
    return -g.numpy()


def advance(X, V, F_fluid, dt, mesh, l0, n_sub=None):
    """Velocity Verlet over one fluid step with a constant fluid force.

    X, V, F_fluid: (nv, 3). Pinned (LE) vertices keep X and V = 0.
    Returns (X, V) at the end of the step.
    """
    n_sub = mesh.substeps(dt) if n_sub is None else n_sub
    h = dt / n_sub
    m = mesh.mass[:, None]
    free = mesh.free[:, None]
    X = X.copy()
    V = V.copy()
    acc = np.where(free, (elastic_forces(X, mesh, l0) + F_fluid) / m, 0.0)
    for _ in range(n_sub):
        V = V + 0.5 * h * acc
        X = X + h * V
        acc = np.where(free, (elastic_forces(X, mesh, l0) + F_fluid) / m, 0.0)
        V = V + 0.5 * h * acc
    V = np.where(free, V, 0.0)
    return X, V
