"""Quantum-jump (MCWF) trajectories and the independent-trajectory Krotov sweep, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Follows, step by step and in the paper's order:

* Sec. 2.1, the MCWF algorithm: propagate under H_eff until ||Psi||^2 = r, jump
  Psi -> L_l Psi / ||L_l Psi|| with channel probability <Psi|L_l^dag L_l|Psi>, draw a new r,
  continue; jump times are located by bisection so several jumps may fall in one step.
* Sec. 2.3, Eq. (independent_traj_update): the sequential Krotov update
      Delta eps_i(t) = S_i(t) / (M lambda_i) sum_k Im <chi_k^(0)(t)| H_i |Psi_k^(1)(t)>
  with chi_k^(0)(T) = tau_k |Psi_tgt> and tau_k the overlap of Eq. (functional_traj).
* Sec. 2.2, Eq. (krotov_functional): J = J_T + sum_i lambda_i/S_i int Delta eps_i^2 dt.
* Sec. 2.3, Eq. (cross_traj_update), the cross-trajectory variant:
      Delta eps_i(t) = S_i(t) / (M^2 lambda_i) sum_{k,k'} Im[<xi_k^(0)(t)|H_i|Psi_k'^(1)(t)> <Psi_k'^(1)(t)|xi_k^(0)(t)>]
  with xi_k^(0)(T) = |Psi_tgt> propagated backward like chi_k (along trajectory k's record).

Readings of points the paper leaves open (each listed with this build's design notes):
the state is not renormalised between jumps and is renormalised after each jump; a jump
happens iff ||psi||^2 <= r; bisection stops when hi - lo <= 2^-48 dt (at most 60 halvings)
and takes s* = hi; the channel is the first l whose cumulative probability reaches
u * sum_l p_l; uniforms come from ``synth_inputs.uniforms`` (column 0 = first r, columns
2m-1 / 2m = channel draw / next r after jump m); the co-state is propagated backward along
each trajectory's own recorded jumps (the exact adjoint of that trajectory's forward map,
applying conj(c) L_l^dag at s*); the update of interval j uses psi^(1)(t_{j-1}),
chi^(0)(t_{j-1}) and S_i(t_{j-1/2}); the final state is normalised for tau_k.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .propagate import StepPropagator

BISECT_REL_TOL = 2.0 ** -48
BISECT_MAX_IT = 60


@dataclass
class Jump:
    step: int       # 1-based interval index j (jump inside [t_{j-1}, t_j])
    s: float        # time offset of the jump from t_{j-1}
    channel: int    # Lindblad operator index l
    c: float        # renormalisation 1 / ||L_l psi(s)||


@dataclass
class ForwardResult:
    psi_T: np.ndarray                 # [M, d] final (unnormalised) states
    records: list                     # per trajectory: list[Jump]
    eps: np.ndarray                   # [n_ctrl, nt] pulse used by this pass
    deps: np.ndarray                  # [n_ctrl, nt] update (zeros without update)
    margin: np.ndarray                # [M] min over interval ends of | ||psi||^2 - r | (incl. those that jump)
    psi_t: np.ndarray = None          # [nt+1, M, d] if requested
    error: str = ""
    deps_scale: np.ndarray = None     # [n_ctrl, nt] magnitude of the summed terms (update only): the
                                      # sum is over trajectories and elements x of Im(conj(chi_kx) (H_i psi_k)_x),
                                      # S/(lambda M) sum_{k,x} |conj(chi_kx) (H_i psi_k)_x|; cross rule:
                                      # S/(lambda M^2) sum_{k,k'} (sum_x |xi_kx||(H_i psi_k')_x|)(sum_x |xi_kx||psi_k'x|)


def _norm2(v: np.ndarray) -> float:
    return float(np.vdot(v, v).real)


class JumpRecordFull(RuntimeError):
    pass


def _step_with_jumps(prop: StepPropagator, Ls: list, psi: np.ndarray, dt: float, j: int,
                     state: dict, u_row: np.ndarray, max_jumps: int, records: list,
                     first_order: bool = False) -> np.ndarray:
    """Advance one trajectory over one interval [t_{j-1}, t_j] with MCWF jumps.

    ``first_order``: the alternative scheme of Sec. 2.1 with at most one jump per time step -- the
    jump found at the end of the interval is applied there (s* = dt), without locating its time.
    """
    s0 = 0.0
    start = psi
    while True:
        phi = prop.apply(start, dt - s0)
        n_end = _norm2(phi)
        # distance of the no-jump norm at the interval's end from the threshold: it decides whether
        # the jump falls in this interval or a later one, whichever way it goes
        state["margin"] = min(state["margin"], abs(n_end - state["r"]))
        if n_end > state["r"]:
            return phi
        # a jump happens in (s0, dt]: locate it by bisection on the norm
        lo, hi = (dt - s0 if first_order else 0.0), dt - s0
        it = 0
        while hi - lo > BISECT_REL_TOL * dt and it < BISECT_MAX_IT:
            mid = 0.5 * (lo + hi)
            if _norm2(prop.apply(start, mid)) <= state["r"]:
                hi = mid
            else:
                lo = mid
            it += 1
        phi = prop.apply(start, hi)
        m = state["jumps"] + 1
        if m > max_jumps:
            raise JumpRecordFull(f"trajectory exceeded {max_jumps} jumps")
        p = np.array([_norm2(l_op @ phi) for l_op in Ls])
        u = u_row[2 * m - 1]
        cum = np.cumsum(p)
        ch = int(np.searchsorted(cum, u * cum[-1], side="left"))
        ch = min(ch, len(Ls) - 1)
        lphi = Ls[ch] @ phi
        nrm = np.sqrt(_norm2(lphi))
        if nrm == 0.0:
            raise RuntimeError("jump into a zero state")
        records.append(Jump(j, s0 + hi, ch, 1.0 / nrm))
        state["jumps"] = m
        state["r"] = float(u_row[2 * m])
        start = lphi / nrm
        s0 = s0 + hi


def cross_overlap(xi: np.ndarray, psi: np.ndarray, Hc: np.ndarray, scale: bool = False):
    """sum_{k,k'} Im[<xi_k|Hc|psi_k'> <psi_k'|xi_k>] for xi, psi [M, d] (Eq. cross_traj_update);
    with scale, also the magnitude of what is summed: sum_{k,k'} of the product of the two inner
    products' element-magnitude sums (the size of the terms before any cancellation)."""
    hpsi = psi @ Hc.T
    A = np.conj(xi) @ hpsi.T                  # A[k, k'] = <xi_k|Hc|psi_k'>
    G = np.conj(xi) @ psi.T                   # G[k, k'] = <xi_k|psi_k'>, so <psi_k'|xi_k> = conj(G)
    terms = np.imag(A * np.conj(G))
    if scale:
        mag = (np.abs(xi) @ np.abs(hpsi).T) * (np.abs(xi) @ np.abs(psi).T)
        return float(np.sum(terms)), float(np.sum(mag))
    return float(np.sum(terms))


def forward_pass(model, eps: np.ndarray, T: float, U_pass: np.ndarray, psi0: np.ndarray,
                 chi: np.ndarray = None, shape: np.ndarray = None, lam: np.ndarray = None,
                 keep_states: bool = False, max_jumps: int = None, cross: bool = False,
                 first_order: bool = False) -> ForwardResult:
    """One forward MCWF sweep over all M trajectories.

    Without ``chi`` the pulse ``eps`` is used as is.  With ``chi`` ([nt+1, M, d], the
    co-states of the previous backward sweep) the Krotov update is applied sequentially:
    before interval j is propagated, Delta eps_ij is formed from all trajectories' states
    at t_{j-1} and the new value eps_ij + Delta eps_ij is used for that interval.
    ``psi0`` is [d] (same initial state for every trajectory) or [M, d].  With ``cross`` the
    co-states are the xi_k of Eq. (cross_traj_update) and the update is the cross-trajectory one.
    """
    n_ctrl, nt = eps.shape
    M = U_pass.shape[0]
    dt = T / nt
    if max_jumps is None:
        max_jumps = (U_pass.shape[1] - 1) // 2
    psi = np.array(np.broadcast_to(psi0, (M, psi0.shape[-1])), dtype=np.complex128)
    eps_used = np.array(eps, dtype=np.float64)
    deps = np.zeros_like(eps_used)
    deps_scale = np.zeros_like(eps_used)
    states = [{"r": float(U_pass[k, 0]), "jumps": 0, "margin": np.inf} for k in range(M)]
    records = [[] for _ in range(M)]
    psi_t = [psi.copy()] if keep_states else None
    Ls = model.L
    for j in range(1, nt + 1):
        if chi is not None:
            for i in range(n_ctrl):
                if cross:
                    g, ga = cross_overlap(chi[j - 1], psi, model.Hc[i], scale=True)
                    deps[i, j - 1] = shape[i, j - 1] / (lam[i] * M * M) * g
                    deps_scale[i, j - 1] = shape[i, j - 1] / (lam[i] * M * M) * ga
                    continue
                hpsi = psi @ model.Hc[i].T          # rows: Hc_i psi_k
                prod = np.conj(chi[j - 1]) * hpsi
                gk = np.imag(np.sum(prod, axis=1))
                g = np.sum(gk)
                deps[i, j - 1] = shape[i, j - 1] / (lam[i] * M) * g
                deps_scale[i, j - 1] = shape[i, j - 1] / (lam[i] * M) * np.sum(np.abs(prod))
            eps_used[:, j - 1] = eps[:, j - 1] + deps[:, j - 1]
        prop = StepPropagator(model.Heff(eps_used[:, j - 1]))
        # every trajectory first takes the full interval; those whose norm fell to the
        # threshold are redone from t_{j-1} with the jump search
        full = prop.apply(psi.T, dt).T
        n_end = np.sum(np.abs(full) ** 2, axis=1)
        new = np.empty_like(psi)
        for k in range(M):
            if n_end[k] > states[k]["r"]:
                states[k]["margin"] = min(states[k]["margin"], n_end[k] - states[k]["r"])
                new[k] = full[k]
            else:
                new[k] = _step_with_jumps(prop, Ls, psi[k], dt, j, states[k], U_pass[k],
                                          max_jumps, records[k], first_order)
        psi = new
        if keep_states:
            psi_t.append(psi.copy())
    return ForwardResult(psi, records, eps_used, deps,
                         np.array([s["margin"] for s in states]),
                         np.array(psi_t) if keep_states else None, deps_scale=deps_scale)


def fidelity(psi_T: np.ndarray, psi_tgt: np.ndarray):
    """tau_k = <Psi_tgt | psi_k(T)/||psi_k(T)||>, F = mean |tau_k|^2 (Eq. functional_traj)."""
    nrm = np.sqrt(np.sum(np.abs(psi_T) ** 2, axis=1))
    tau = (psi_T.conj() @ psi_tgt).conj() / nrm   # <tgt|psi> = conj(<psi|tgt>)
    return tau, float(np.mean(np.abs(tau) ** 2))


def backward_pass(model, eps: np.ndarray, T: float, chi_T: np.ndarray, records: list) -> np.ndarray:
    """Co-states chi_k(t_j), j = nt..0, under pulse ``eps`` along each trajectory's record.

    chi_k(t_{j-1}) = U_kj^dag chi_k(t_j), where U_kj is trajectory k's forward map over
    interval j: free propagation pieces expm(-i H_eff tau) separated by the recorded jumps
    c L_l.  Returns an array [nt+1, M, d].
    """
    n_ctrl, nt = eps.shape
    M, d = chi_T.shape
    dt = T / nt
    by_step = {}
    for k, recs in enumerate(records):
        for rec in recs:
            by_step.setdefault((rec.step, k), []).append(rec)
    out = np.empty((nt + 1, M, d), dtype=np.complex128)
    out[nt] = chi_T
    for j in range(nt, 0, -1):
        prop = StepPropagator(model.Heff(eps[:, j - 1]))
        cur = out[j]
        nxt = prop.apply_adjoint(cur.T, dt).T      # trajectories without a jump in interval j
        for k in range(M):
            if (j, k) not in by_step:
                continue
            recs = sorted(by_step[(j, k)], key=lambda r: r.s)
            chi = cur[k]
            t_hi = dt
            for rec in reversed(recs):
                chi = prop.apply_adjoint(chi, t_hi - rec.s)
                chi = np.conj(rec.c) * (model.L[rec.channel].conj().T @ chi)
                t_hi = rec.s
            nxt[k] = prop.apply_adjoint(chi, t_hi)
        out[j - 1] = nxt
    return out


def krotov_functional(JT: float, deps: np.ndarray, shape: np.ndarray, lam: np.ndarray, dt: float) -> float:
    """J = J_T + sum_i lambda_i sum_j Delta eps_ij^2 dt / S_ij (points with S = 0 excluded)."""
    mask = shape > 0
    ratio = np.zeros_like(deps)
    ratio[mask] = deps[mask] ** 2 / shape[mask]
    return float(JT + np.sum(lam[:, None] * ratio) * dt)


@dataclass
class OptimizationResult:
    eps: np.ndarray
    JT: list = field(default_factory=list)       # J_T after each forward pass (pass 0 = guess)
    J: list = field(default_factory=list)        # J after each updating pass
    forward: list = field(default_factory=list)  # ForwardResult of each pass (if kept)
    chi: list = field(default_factory=list)      # co-states of each backward sweep (if kept)


def optimize(model, eps0: np.ndarray, T: float, U: np.ndarray, shape: np.ndarray, lam: np.ndarray,
             n_iter: int, psi0=None, keep: bool = False, update: str = "independent",
             first_order: bool = False) -> OptimizationResult:
    """Trajectory Krotov: guess pass 0, then n_iter x [backward; updating forward].

    Forward pass p reads uniforms U[p]; iteration n uses the records of pass n-1.  ``update``:
    "independent" (Eq. independent_traj_update, chi_k(T) = tau_k |tgt>) or "cross"
    (Eq. cross_traj_update, xi_k(T) = |tgt>).
    """
    cross = update == "cross"
    psi0 = model.psi0 if psi0 is None else psi0
    nt = eps0.shape[1]
    dt = T / nt
    fw = forward_pass(model, eps0, T, U[0], psi0, first_order=first_order)
    tau, F = fidelity(fw.psi_T, model.psi_tgt)
    res = OptimizationResult(eps=eps0.copy(), JT=[1.0 - F])
    if keep:
        res.forward.append(fw)
    eps = eps0.copy()
    for n in range(1, n_iter + 1):
        boundary = np.ones_like(tau) if cross else tau
        chi = backward_pass(model, eps, T, boundary[:, None] * model.psi_tgt[None, :], fw.records)
        fw = forward_pass(model, eps, T, U[n], psi0, chi=chi, shape=shape, lam=lam, cross=cross,
                          first_order=first_order)
        eps = fw.eps
        tau, F = fidelity(fw.psi_T, model.psi_tgt)
        res.JT.append(1.0 - F)
        res.J.append(krotov_functional(1.0 - F, fw.deps, shape, lam, dt))
        if keep:
            res.forward.append(fw)
            res.chi.append(chi)
    res.eps = eps
    return res
