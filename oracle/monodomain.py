"""Crank-Nicolson step of the PolyDG monodomain + Barreto-Cressman model (FP64).

Eq. fully-discrete-1 of the paper:
    K_h U^{k+1} = (chi_m C_m M_h - dt/2 A_h) U^k - chi_m dt I^{k+1} + dt F^{k+1},
with the ionic state advanced explicitly.  Readings (listed with the others):
  * the ionic state lives at the element quadrature nodes and is advanced
    by explicit Euler with u^k at the node: y^{k+1} = y^k - dt m(u^k, y^k);
  * I^{k+1}_i = sum_q w_q f(u~_q, y^{k+1}_q) phi_i(x_q), where
    u~ = 3/2 U^k - 1/2 U^{k-1} is the second-order extrapolation to the
    Crank-Nicolson midpoint (u~ = U^0 on the first step);
  * F^{k+1}_i = int I_ext(x, t^{k+1/2}) phi_i with the Gaussian stimulus
    I_ext = A exp(-|x - x0|^2 / (2 w^2)) switched on while t < duration;
  * chi_m C_m = chi_cm and C_m = 1, so chi_m = chi_cm;
  * ionic_form="modal" takes the second line of Eq. fully-discrete-1 as printed
    instead: per state l the DG coefficients Y_l, M_h Y_l^{k+1} = M_h Y_l^k - dt G_l^k
    with G_l = int m_l(u_h^k, y_h^k) phi (element quadrature), so
    Y_l^{k+1} = Y_l^k + M_K^{-1} sum_q w_q dt y'_l(x_q) phi(x_q) cell by cell, and
    I^{k+1} uses y_h^{k+1} at the nodes.  The initial state is the rest state as a
    constant (coefficient of the constant mode, phi_0 = 1).
The linear solve is either a direct sparse factorisation (the definition:
the method's PCG converges to that solution) or PCG with B_ad (Eq. prec).

Pins (tests/test_oracle_monodomain.py): with f = 0 and no stimulus the
scheme conserves int u (Neumann) exactly; on a single eigenmode of the
generalised problem A v = lambda M v the amplification factor is
(1 - dt lambda/2)/(1 + dt lambda/2).  The ion term (tests/test_oracle_ionic.py):
a linear current g u on an eigenmode follows the closed-form two-step recurrence
(chi + dt lambda/2) a_{k+1} = (chi - dt lambda/2) a_k - chi dt g u~_k; an affine
current on the constant mode and a current of the updated state likewise; with a
frozen state a uniform field converges at second order in dt to the exact solution
of u' = -f(u), and with the explicit state update at first order; the stimulus
enters as dt F while t^{k+1/2} < duration.
"""
from dataclasses import dataclass

import numpy as np
import scipy.sparse.linalg as spla

from . import basis, ionic
from .assembly import element_rule, load_vector
from .pcg import pcg


@dataclass
class Nodes:
    cell: np.ndarray      # [nn] element of each node
    x: np.ndarray         # [nn, dim]
    w: np.ndarray         # [nn]
    phi: np.ndarray       # [nn, n_p] basis values of the node's element


def quadrature_nodes(disc) -> Nodes:
    cells, xs, ws, phis = [], [], [], []
    for k in range(disc.mesh.n_cells):
        x, w = element_rule(disc.mesh, k, disc.p)
        V, _ = basis.eval_basis(disc.p, disc.geom.bbox[k], x)
        cells.append(np.full(len(w), k)); xs.append(x); ws.append(w); phis.append(V)
    return Nodes(np.concatenate(cells), np.concatenate(xs), np.concatenate(ws),
                 np.concatenate(phis))


def nodal_values(nodes: Nodes, U, n_p):
    """u(x_q) = sum_j U_{K(q), j} phi_j(x_q)."""
    return np.einsum("qj,qj->q", nodes.phi, U.reshape(-1, n_p)[nodes.cell])


def project_nodal(nodes: Nodes, g, n_cells, n_p):
    """b_{K,i} = sum_{q in K} w_q g_q phi_i(x_q)."""
    out = np.zeros((n_cells, n_p))
    np.add.at(out, nodes.cell, (nodes.w * g)[:, None] * nodes.phi)
    return out.ravel()


def stimulus_load(disc, stim):
    """Spatial profile int A exp(-|x-x0|^2/(2w^2)) phi_i (time switch applied by the caller)."""
    A, w = stim["amplitude"], stim["width"]
    x0 = np.array([stim["x0"], stim["y0"]] + ([stim["z0"]] if disc.mesh.dim == 3 else []))
    return load_vector(disc, lambda x: A * np.exp(-((x - x0) ** 2).sum(1) / (2.0 * w * w)))


@dataclass
class State:
    U: np.ndarray
    U_prev: np.ndarray
    y: np.ndarray          # [5, nn] the states at the nodes
    k: int = 0
    Y: np.ndarray = None   # [5, n_dofs] DG coefficients of the states (modal form)


class Monodomain:
    def __init__(self, disc, stimulus, u0=-67.0, solver="direct", prec=None, rtol=1e-8,
                 flexible=False, ion=True, ionic_form="nodal"):
        self.disc = disc
        self.nodes = quadrature_nodes(disc)
        self.stim = stimulus
        self.F = stimulus_load(disc, stimulus) if stimulus else np.zeros(disc.n_dofs)
        self.Kminus = (disc.chi_cm * disc.M - (0.5 * disc.dt) * disc.A).tocsr()
        self.solver, self.prec, self.rtol, self.flexible = solver, prec, rtol, flexible
        self.ion = ion
        self.lu = spla.splu(disc.K.tocsc()) if solver == "direct" else None
        U0 = np.zeros(disc.n_dofs)
        U0[::disc.n_p] = u0                      # constant u0: only the (0,0) mode
        rest = ionic.rest_state(u0)
        y0 = np.repeat(rest[:, None], len(self.nodes.w), axis=1)
        self.ionic_form = ionic_form
        Y0 = None
        if ionic_form == "modal":
            Y0 = np.zeros((5, disc.n_dofs))
            Y0[:, ::disc.n_p] = rest[:, None]
        elif ionic_form != "nodal":
            raise ValueError(ionic_form)
        self.state = State(U0, U0.copy(), y0, 0, Y0)
        self.iterations = []

    def rhs(self, st: State):
        d = self.disc
        dt = d.dt
        u_nodes = nodal_values(self.nodes, st.U, d.n_p)
        Y_new = None
        if self.ionic_form == "modal":
            Y_new = self.modal_update(u_nodes, st.Y)
            y_new = np.stack([nodal_values(self.nodes, Y_new[l], d.n_p) for l in range(5)])
        else:
            y_new = ionic.euler_step(u_nodes, st.y, dt)
        U_ext = st.U if st.k == 0 else 1.5 * st.U - 0.5 * st.U_prev
        if self.ion:
            f = ionic.f_ion(nodal_values(self.nodes, U_ext, d.n_p), y_new)
            I = project_nodal(self.nodes, f, d.mesh.n_cells, d.n_p)
        else:
            I = np.zeros(d.n_dofs)
        t_half = (st.k + 0.5) * dt
        on = 1.0 if (self.stim and t_half < self.stim["duration"]) else 0.0
        b = self.Kminus @ st.U - d.chi_cm * dt * I + dt * on * self.F
        self._Y_new = Y_new
        return b, y_new

    def modal_update(self, u_nodes, Y):
        """Y_l + M_K^{-1} sum_q w_q dt y'_l(u^k(x_q), y_h^k(x_q)) phi(x_q), cell by cell."""
        d, nc, n_p = self.disc, self.disc.mesh.n_cells, self.disc.n_p
        yq = np.stack([nodal_values(self.nodes, Y[l], n_p) for l in range(5)])
        incr = d.dt * ionic.dydt(u_nodes, yq)
        out = np.empty_like(Y)
        for l in range(5):
            G = project_nodal(self.nodes, incr[l], nc, n_p).reshape(nc, n_p, 1)
            out[l] = Y[l] + np.linalg.solve(d.M_blocks, G).ravel()
        return out

    def step(self):
        st = self.state
        b, y_new = self.rhs(st)
        if self.solver == "direct":
            U_new = self.lu.solve(b)
            self.iterations.append(0)
        else:
            res = pcg(self.disc.K, b, x0=st.U, prec=self.prec, rtol=self.rtol,
                      flexible=self.flexible)
            U_new = res.x
            self.iterations.append(res.iterations)
        self.state = State(U_new, st.U, y_new, st.k + 1, self._Y_new)
        return self.state
