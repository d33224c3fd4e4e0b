"""Generic FP64 Levenberg-Marquardt over a hypergraph of vertex and edge sets (oracle).

Test infrastructure only.  Follows Sec. II:
  cost      F(x) = 1/2 sum_e rho(s_e),  s_e = r_e^T Omega_e r_e            (Eq. 1, Eq. 7)
  linearise r(x + dx) ~ r + J dx                                          (Eq. 3)
  step      argmin 1/2 |r + J dx|^2_W + lambda/2 |D dx|^2                  (Eq. 4)
  normal    (J^T W J + lambda D^T D) dx = -J^T W r,  i.e. H_lambda dx = -b (Eq. 5-6)
with these readings where the paper is silent:
  * D^T D = clamp(diag(H), diag_min, diag_max) (Marquardt, with the Hessian-diagonal
    clamping of Sec. IV-E), or the identity (the other choice Eq. 4 allows);
  * W: Huber first-order weights rho'(s_e) (Eq. 7), whitening by Omega = U^T U;
  * the step is solved exactly: the eliminated vertex sets (points) are removed by a
    Schur complement formed densely, the reduced system is factorised by dense
    Cholesky, and the eliminated unknowns are back-substituted;
  * gain ratio rho = (F(x) - F(x + dx)) / (L(0) - L(dx)) with the model decrease
    L(0) - L(dx) = -b^T dx - 1/2 sum_e |J_e dx|^2_W;
  * acceptance and damping follow Nielsen's rule: accept iff L(0) - L(dx) > 0,
    F(x + dx) is finite and F(x + dx) < F(x) (a reduced system that the Cholesky factorisation
    finds not positive definite counts as a rejected step, as in Ceres);
    then lambda *= max(1/3, 1 - (2 rho - 1)^3),
    nu = 2; otherwise lambda *= nu, nu *= 2; lambda is then clamped to
    [lambda_min, lambda_max] (1e-16, 1e32 by default, the inverse trust-region radius
    bounds of Ceres, which Sec. IV-E follows for its clamping).  Exactly max_iters iterations run
    (accepted or not), as the paper's `iterations` option implies (Listing 5).
Fixed vertices (Listing 5, set_fixed) have no unknowns; inactive edges (set_active)
contribute neither rows nor cost.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable

import numpy as np
import scipy.linalg
import scipy.sparse as sp

from . import robust


@dataclass
class VertexSet:
    name: str
    dim: int                       # tangent-space dimension
    state: np.ndarray              # (n, state_size) float64
    retract: Callable              # (state rows, delta rows) -> new state rows
    eliminate: bool = False        # Schur-eliminated (points)
    fixed: np.ndarray | None = None

    def __post_init__(self):
        self.state = np.array(self.state, dtype=np.float64, copy=True)
        if self.fixed is None:
            self.fixed = np.zeros(self.state.shape[0], dtype=bool)


@dataclass
class EdgeSet:
    name: str
    slots: list                    # vertex-set names, one per vertex of the edge
    idx: np.ndarray                # (n, len(slots)) vertex indices
    evaluate: Callable             # (list of state rows, data) -> (r (n,m), [J_i (n,m,d_i)])
    data: object = None
    sqrt_info: np.ndarray | None = None   # (n, m, m) U with U^T U = Omega; None = identity
    loss: tuple | None = None      # None or ("huber", delta)
    active: np.ndarray | None = None

    def __post_init__(self):
        self.idx = np.asarray(self.idx).reshape(len(self.idx), -1)
        if self.active is None:
            self.active = np.ones(self.idx.shape[0], dtype=bool)


@dataclass
class Problem:
    vertices: dict
    edges: list

    def copy(self) -> "Problem":
        vs = {k: VertexSet(v.name, v.dim, v.state.copy(), v.retract, v.eliminate, v.fixed.copy())
              for k, v in self.vertices.items()}
        return Problem(vs, list(self.edges))


@dataclass
class LMParams:
    initial_damping: float = 1e-4
    diag_min: float = 1e-6
    diag_max: float = 1e32
    lambda_min: float = 1e-16
    lambda_max: float = 1e32
    damping: str = "marquardt"     # or "identity"


@dataclass
class Report:
    initial_cost: float
    final_cost: float
    iterations: int
    accepted: int
    final_lambda: float
    history: list = field(default_factory=list)


# ---------------------------------------------------------------- evaluation

def _edge_states(problem: Problem, es: EdgeSet, states=None):
    st = states if states is not None else {k: v.state for k, v in problem.vertices.items()}
    act = es.active
    return [st[name][es.idx[act, i]] for i, name in enumerate(es.slots)], act


def _whiten(es: EdgeSet, r, Js, act):
    if es.sqrt_info is None:
        return r, Js
    U = es.sqrt_info[act]
    return np.einsum("nij,nj->ni", U, r), [U @ J for J in Js]


def edge_costs(problem: Problem, states=None) -> list:
    """Per edge set: rho(s_e) / 2 for the active edges."""
    out = []
    for es in problem.edges:
        xs, act = _edge_states(problem, es, states)
        data = es.data[act] if isinstance(es.data, np.ndarray) and es.data.ndim > 0 else es.data
        r, Js = es.evaluate(xs, data)
        rw, _ = _whiten(es, r, Js, act)
        s = np.sum(rw * rw, axis=1)
        out.append(0.5 * robust.rho(s, es.loss))
    return out


def total_cost(problem: Problem, states=None) -> float:
    """F(x) = 1/2 sum_e rho(s_e) (Eq. 1 with Eq. 7)."""
    return float(sum(c.sum() for c in edge_costs(problem, states)))


# ---------------------------------------------------------------- layout

@dataclass
class Layout:
    """Column offsets of the free vertices: reduced sets first, eliminated sets after."""
    offsets: dict          # name -> (n,) int offsets, -1 for fixed
    n_reduced: int
    n_total: int
    elim_dim: int          # tangent dimension of the eliminated blocks (0 if none)


def make_layout(problem: Problem) -> Layout:
    offs = {}
    col = 0
    order = [v for v in problem.vertices.values() if not v.eliminate] + \
            [v for v in problem.vertices.values() if v.eliminate]
    n_red = None
    elim_dims = set()
    for v in order:
        if v.eliminate and n_red is None:
            n_red = col
        free = ~v.fixed
        o = -np.ones(v.state.shape[0], dtype=np.int64)
        o[free] = col + v.dim * np.arange(int(free.sum()))
        col += v.dim * int(free.sum())
        offs[v.name] = o
        if v.eliminate:
            elim_dims.add(v.dim)
    if n_red is None:
        n_red = col
    assert len(elim_dims) <= 1, "eliminated vertex sets must share one block size"
    return Layout(offs, n_red, col, elim_dims.pop() if elim_dims else 0)


# ---------------------------------------------------------------- linearisation

@dataclass
class Linearization:
    J: sp.csr_matrix          # weighted, whitened Jacobian (rows x n_total)
    r: np.ndarray             # weighted, whitened residual
    cost: float


def linearize(problem: Problem, layout: Layout) -> Linearization:
    rows, cols, vals, rs = [], [], [], []
    row0 = 0
    cost = 0.0
    for es in problem.edges:
        xs, act = _edge_states(problem, es)
        data = es.data[act] if isinstance(es.data, np.ndarray) and es.data.ndim > 0 else es.data
        r, Js = es.evaluate(xs, data)
        rw, Jw = _whiten(es, r, Js, act)
        s = np.sum(rw * rw, axis=1)
        cost += 0.5 * float(robust.rho(s, es.loss).sum())
        sw = np.sqrt(robust.weight(s, es.loss))
        rw = rw * sw[:, None]
        n, m = rw.shape
        idx = es.idx[act]
        for i, name in enumerate(es.slots):
            Ji = Jw[i] * sw[:, None, None]
            d = Ji.shape[2]
            off = layout.offsets[name][idx[:, i]]
            free = off >= 0
            e_ids = np.nonzero(free)[0]
            rr = row0 + e_ids[:, None, None] * m + np.arange(m)[None, :, None]
            cc = off[free][:, None, None] + np.arange(d)[None, None, :]
            rows.append(np.broadcast_to(rr, (len(e_ids), m, d)).reshape(-1))
            cols.append(np.broadcast_to(cc, (len(e_ids), m, d)).reshape(-1))
            vals.append(Ji[free].reshape(-1))
        rs.append(rw.reshape(-1))
        row0 += n * m
    J = sp.csr_matrix((np.concatenate(vals) if vals else np.zeros(0),
                       (np.concatenate(rows) if rows else np.zeros(0, int),
                        np.concatenate(cols) if cols else np.zeros(0, int))),
                      shape=(row0, layout.n_total))
    return Linearization(J, np.concatenate(rs) if rs else np.zeros(0), cost)


def normal_equations(lin: Linearization):
    """H = J^T W J and b = J^T W r (Eq. 5-6) from the weighted, whitened rows."""
    H = (lin.J.T @ lin.J).tocsr()
    b = lin.J.T @ lin.r
    return H, np.asarray(b).reshape(-1)


def damping_diagonal(H: sp.spmatrix, params: LMParams) -> np.ndarray:
    """D^T D of Eq. 4: clamp(diag(H), diag_min, diag_max), or ones for identity damping."""
    if params.damping == "identity":
        return np.ones(H.shape[0])
    return np.clip(H.diagonal(), params.diag_min, params.diag_max)


# ---------------------------------------------------------------- linear solves

def _elim_blocks(Hee: sp.spmatrix, d: int) -> np.ndarray:
    n = Hee.shape[0] // d
    B = np.zeros((n, d, d))
    coo = Hee.tocoo()
    assert np.all(coo.row // d == coo.col // d), "eliminated blocks must not couple"
    np.add.at(B, (coo.row // d, coo.row % d, coo.col % d), coo.data)
    return B


def schur_solve(Hl: sp.spmatrix, b: np.ndarray, layout: Layout):
    """Exact solution of Hl dx = -b by eliminating the point blocks.

    S = H_rr - H_re H_ee^-1 H_er   (formed densely, block by block)
    g = -b_r + H_re H_ee^-1 b_e
    S dx_r = g  (dense Cholesky);   dx_e = H_ee^-1 (-b_e - H_er dx_r)
    Returns (dx, S, g)."""
    nr, nt, d = layout.n_reduced, layout.n_total, layout.elim_dim
    Hl = sp.csr_matrix(Hl)
    Hrr = Hl[:nr, :nr].toarray()
    br, be = b[:nr], b[nr:]
    if nt == nr:
        S, g = Hrr, -br
        dxr = scipy.linalg.cho_solve(scipy.linalg.cho_factor(S), g) if nr else np.zeros(0)
        return dxr, S, g
    Hre = Hl[:nr, nr:]
    B = _elim_blocks(Hl[nr:, nr:], d)
    Binv = np.linalg.inv(B)
    ne = B.shape[0]
    Einv = sp.bsr_matrix((Binv, np.arange(ne), np.arange(ne + 1)), shape=(nt - nr, nt - nr)).tocsr()
    S = Hrr - (Hre @ Einv @ Hre.T).toarray() if nr else np.zeros((0, 0))
    g = -br + Hre @ (Einv @ be)
    dxr = scipy.linalg.cho_solve(scipy.linalg.cho_factor(S), g) if nr else np.zeros(0)
    dxe = Einv @ (-be - Hre.T @ dxr)
    return np.concatenate([dxr, dxe]), S, g


def dense_solve(Hl: sp.spmatrix, b: np.ndarray) -> np.ndarray:
    """Brute force: dense solve of the full damped normal equations Hl dx = -b."""
    A = Hl.toarray() if sp.issparse(Hl) else np.asarray(Hl)
    return np.linalg.solve(A, -b)


def model_decrease(lin: Linearization, b: np.ndarray, dx: np.ndarray) -> float:
    """L(0) - L(dx) = -b^T dx - 1/2 |J dx|^2 (weighted, whitened)."""
    Jdx = lin.J @ dx
    return float(-b @ dx - 0.5 * Jdx @ Jdx)


# ---------------------------------------------------------------- update

def apply_step(problem: Problem, layout: Layout, dx: np.ndarray) -> dict:
    """New states x [+] dx; fixed vertices are returned unchanged (bit for bit)."""
    out = {}
    for name, v in problem.vertices.items():
        off = layout.offsets[name]
        free = off >= 0
        new = v.state.copy()
        if np.any(free):
            d = dx[off[free][:, None] + np.arange(v.dim)[None, :]]
            new[free] = v.retract(v.state[free], d)
        out[name] = new
    return out


def nielsen_update(lam: float, nu: float, rho: float, accepted: bool):
    """Damping update: accepted -> lambda * max(1/3, 1 - (2 rho - 1)^3), nu = 2;
    rejected -> lambda * nu, nu * 2."""
    if accepted:
        return lam * max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3), 2.0
    return lam * nu, nu * 2.0


def clamp_lambda(lam: float, params: LMParams) -> float:
    """The damping after each update is kept in [lambda_min, lambda_max]."""
    return min(max(lam, params.lambda_min), params.lambda_max)


def levenberg_marquardt(problem: Problem, max_iters: int, params: LMParams | None = None):
    """Runs exactly max_iters LM iterations on a copy of `problem`; returns (problem, Report)."""
    params = params or LMParams()
    prob = problem.copy()
    layout = make_layout(prob)
    lam, nu = params.initial_damping, 2.0
    F = total_cost(prob)
    rep = Report(F, F, 0, 0, lam)
    for it in range(max_iters):
        lin = linearize(prob, layout)
        H, b = normal_equations(lin)
        D = damping_diagonal(H, params)
        Hl = H + sp.diags(lam * D)
        try:
            dx, _, _ = schur_solve(Hl, b, layout)
        except np.linalg.LinAlgError:
            dx = None                    # reduced system not positive definite at this damping
        if dx is None:
            L, Fc, cand = 0.0, np.inf, None
        else:
            L = model_decrease(lin, b, dx)
            cand = apply_step(prob, layout, dx)
            Fc = total_cost(prob, cand)
        accepted = bool(L > 0 and np.isfinite(Fc) and Fc < F)
        rho = (F - Fc) / L if L != 0 else 0.0
        rep.history.append(dict(iter=it, cost=F, cand_cost=Fc, model_decrease=L, rho=rho,
                                lam=lam, accepted=accepted))
        if accepted:
            for name, st in cand.items():
                prob.vertices[name].state = st
            F = Fc
            rep.accepted += 1
        lam, nu = nielsen_update(lam, nu, rho, accepted)
        lam = clamp_lambda(lam, params)
        rep.iterations += 1
    rep.final_cost = F
    rep.final_lambda = lam
    return prob, rep


def step(problem: Problem, lam: float, params: LMParams | None = None):
    """One damped step at the current state (no acceptance test): returns
    (dx, layout, H, b, D, lin)."""
    params = params or LMParams()
    layout = make_layout(problem)
    lin = linearize(problem, layout)
    H, b = normal_equations(lin)
    D = damping_diagonal(H, params)
    dx, _, _ = schur_solve(H + sp.diags(lam * D), b, layout)
    return dx, layout, H, b, D, lin


# ---------------------------------------------------------------- problem builders

def ba_problem(cams, pts, cam_idx, pt_idx, obs, huber_delta=None, cam_fixed=None,
               pt_fixed=None, active=None, sqrt_info=None) -> Problem:
    """Bundle-adjustment problem (cameras reduced, points eliminated)."""
    from . import ba
    vs = {
        "cam": VertexSet("cam", 9, cams, ba.retract_cams, False, cam_fixed),
        "pt": VertexSet("pt", 3, pts, ba.retract_points, True, pt_fixed),
    }
    loss = None if huber_delta is None else ("huber", float(huber_delta))
    es = EdgeSet("reproj", ["cam", "pt"], np.stack([cam_idx, pt_idx], axis=1), ba.evaluate,
                 np.asarray(obs, dtype=np.float64), sqrt_info, loss, active)
    return Problem(vs, [es])
