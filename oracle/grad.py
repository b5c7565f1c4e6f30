"""O3 -- gradients of the measured probability through the mapped RK4 solve (oracle).

Loss: l = Re Tr(rho0 A(T)) with A(T) from O2 (oracle.mapping), i.e. for every initial
condition, l = Re sum_IC w sum_{k,l} rho0_{l,k} sqrt(k! l!) (G_x[k] G_y[l] + R[k,l])
(Eq. 7 with T_{k,l} = sqrt(k! l!)|k><l|).

Parameters: the real H-term parameters theta_p (terms with ``param = p``; their
coefficient is coef * theta_p, and theta also enters the separation constant of Eq. 304
through omega_j, eta_j) and the real and imaginary parts of every segment of every
piecewise-constant channel.

Method: the exact discrete adjoint of classical RK4 applied to the separated system of
Eqs. 9a-c (with the secular dissipator's projector P of Eq. 302c where the problem has one:
P^T acts on b_R and, through the source P(G_x G_y), on G_x and G_y).  With stage inputs u_i, stage derivatives k_i = f(u_i, t_i) and
z' = z + h/6 (k1 + 2 k2 + 2 k3 + k4), the cotangent lam' of z' is pulled back as
    b4 = h/6 lam',  q_i = J_i^T b_i,  b3 = h/3 lam' + h q4,  b2 = h/3 lam' + h/2 q3,
    b1 = h/6 lam' + h/2 q2,  lam = lam' + q1 + q2 + q3 + q4,
    dl/dtheta += Re sum_i <b_i, df/dtheta(u_i, t_i)>,
with <.,.> the bilinear (unconjugated) pairing: the system is complex-linear in its state.
J^T of the bilinear source S(G_x G_y) contributes to G_x and G_y.  Forward states are
checkpointed every ``checkpoint_every`` steps and each segment is recomputed once.

Diagonal residual layout (``r_layout="diag"``, the R(xy) reading of oracle.mapping): the R
equation is projected onto its diagonal k = l, dR = D(f_R), and R stays diagonal.  D is
symmetric under the bilinear pairing, so J^T acts on D(b_R) and its R component is projected
again; the cotangent of the final R is D(dl/dG).

The number-basis method (O1, oracle.fock) has its own discrete adjoint,
``loss_and_grad_direct``: the same RK4 pull-back with the transposed generator of Eq. 3
(every product X A Y becomes X^T B Y^T under the bilinear pairing).

Parity status: pinned by central finite differences of oracle.mapping.rk4_mapped
(tests/test_oracle_grad.py), with conventional jump operators and with the secular
dissipator (one and two modes, finite temperature), in the full and the diagonal residual
layouts; ``loss_and_grad_direct`` by central finite differences of oracle.fock.rk4_adjoint
(one and two modes, thermal jump operators and the secular dissipator).
"""

from __future__ import annotations

import math
from typing import Dict, List, Optional, Sequence

import numpy as np

from workloads.spec import Problem
from .channels import stage_value
from .fock import _max_degree, kron_restricted
from .mapping import MappedModel, left_factors, map_initial, omega_eta, right_factors, separation_constant

RK_C = (0.0, 0.5, 0.5, 1.0)


def _seed(problem: Problem, M) -> np.ndarray:
    """dl/dG[k, l] = rho0_{l,k} sqrt(k! l!) (flattened x, y indices)."""
    n = problem.n_modes
    d = int(np.prod(M))
    lam = np.zeros((d, d), dtype=np.complex128)
    for (k, l), r in problem.rho0_items().items():
        if all(a < m for a, m in zip(k, M)) and all(b < m for b, m in zip(l, M)):
            # Tr(rho0 A) = sum <k|rho0|l> <l|A|k>: the A element is (l, k)
            kk = int(np.ravel_multi_index(l, M))
            ll = int(np.ravel_multi_index(k, M))
            fac = math.sqrt(math.prod(math.factorial(x) for x in l) * math.prod(math.factorial(x) for x in k))
            lam[kk, ll] += r * fac
    del n
    return lam


class _Derivs:
    """df/dtheta pieces: per H term its left / right matrices (restricted) and coefficient."""

    def __init__(self, problem: Problem, model: MappedModel):
        self.p = problem
        pad = 2 * _max_degree(problem) + 2
        big = tuple(m + pad for m in model.M)
        self.terms = []  # (left, right, coef_without_theta, param, channel, conj)
        for t in problem.h_terms:
            if t.param < 0 and t.channel < 0:
                continue
            lo = kron_restricted(left_factors(t.u, t.v, big), model.M)
            ro = kron_restricted(right_factors(t.u, t.v, big), model.M)
            self.terms.append((lo, ro, complex(t.coef), t.param, t.channel, t.conj))
        self.n_params = len(problem.params)

    def dC(self, p_idx, q_idx) -> List[complex]:
        """dC/dtheta_p of Eq. 304 for the IC (p, q)."""
        out = [0j] * self.n_params
        for t in self.p.h_terms:
            if t.param < 0 or t.channel >= 0:
                continue
            nz = [j for j in range(self.p.n_modes) if t.u[j] or t.v[j]]
            if len(nz) != 1:
                continue
            j = nz[0]
            c = complex(t.coef).real
            pj, qj = p_idx[j], q_idx[j]
            if t.u[j] == 1 and t.v[j] == 1:
                out[t.param] += -0.5j * c * (pj + qj)
            elif t.u[j] == 2 and t.v[j] == 2:
                out[t.param] += -0.5j * c * (pj * pj + qj * qj - pj - qj)
        return out


def loss_and_grad(problem: Problem, M: Optional[Sequence[int]] = None, checkpoint_every: int = 64,
                  r_layout: str = "full"):
    """Returns (loss, dl/dtheta (len P), {channel: dl/d(Re, Im) of each segment (n_seg, 2)}).
    r_layout: "full" (Eq. 303c) or "diag" (R kept on k = l, as in oracle.mapping)."""
    if r_layout not in ("full", "diag"):
        raise ValueError(f"r_layout {r_layout!r}")
    diag = r_layout == "diag"
    proj = (lambda X: np.diag(np.diag(X))) if diag else (lambda X: X)
    model = MappedModel(problem, M)
    M = model.M
    der = _Derivs(problem, model)
    p = problem
    dt = p.dt
    steps = p.n_steps
    g0, ics = map_initial(problem, M)
    lamG = _seed(problem, M)
    d = model.dim
    grad_theta = np.zeros(len(p.params))
    grad_pwc: Dict[int, np.ndarray] = {}
    for ci, ch in enumerate(p.channels):
        if ch.kind == "pwc":
            grad_pwc[ci] = np.zeros(((len(ch.params) - 2) // 2, 2))
    loss = 0.0

    def ops(tau, c):
        return model.operators(tau, c, dt)

    def f(z, O, C):
        return model.rhs(z[0], z[1], z[2], O[0], O[1], C, r_layout)

    def JT(b, u, O, C):
        """Transpose of df/dz at u applied to b = (b_gx, b_gy, b_R)."""
        bx, by, bR = b
        bR = proj(bR)
        Ox, Oy = O
        qx = Ox.T @ bx + C * bx
        qy = Oy.T @ by - C * by
        qR = Ox.T @ bR + bR @ Oy
        for kappa, Ld_l, L_r in model.sandwich:
            qR += kappa * (Ld_l.T @ bR @ L_r)
            # source kappa (Ld_l gx) (L_r gy)^T: derivative wrt gx and gy
            qx += kappa * (Ld_l.T @ (bR @ (L_r @ u[1])))
            qy += kappa * (L_r.T @ (bR.T @ (Ld_l @ u[0])))
        if model.secular:
            # secular projector P on R and on the source P(G_x G_y) (Eq. 303c with Eq. 302c)
            PT = model.secular_projector_T(bR)
            qR += PT
            qx += PT @ u[1]
            qy += PT.T @ u[0]
        return qx, qy, proj(qR)

    def param_dot(b, u, tau_step, c, C_derivs):
        """Adds Re <b, df/dtheta(u)> for every parameter and pwc segment."""
        bx, by, bR = b
        bR = proj(bR)
        ux, uy, uR = u
        for lo, ro, coef, param, chn, conj in der.terms:
            # action of d(Ox)/dh and d(Oy)/dh for this term (h = coef * theta * chan)
            act = np.sum(bx * (1j * lo @ ux)) + np.sum(by * (-1j * ro @ uy)) \
                + np.sum(bR * (1j * lo @ uR + uR @ (-1j * ro).T))
            theta = p.params[param] if param >= 0 else 1.0
            e = 1.0 + 0j
            if chn >= 0:
                e = stage_value(p.channels[chn], tau_step, c, dt, p.T, p.reverse_time)
                e = np.conj(e) if conj else e
            if param >= 0:
                grad_theta[param] += (coef * e * act).real
            if chn >= 0 and p.channels[chn].kind == "pwc":
                chd = p.channels[chn]
                tt = (p.T - (tau_step + 0.5 * dt)) if p.reverse_time else tau_step + 0.5 * dt
                s = int(math.floor((tt - chd.params[0]) / chd.params[1]))
                if 0 <= s < grad_pwc[chn].shape[0]:
                    g = coef * theta * act
                    grad_pwc[chn][s, 0] += g.real
                    grad_pwc[chn][s, 1] += (g * (-1j if conj else 1j)).real
        for pi, dc in enumerate(C_derivs):
            if dc != 0:
                grad_theta[pi] += (dc * (np.sum(bx * ux) - np.sum(by * uy))).real

    for (pp, qq, w) in ics:
        C = separation_constant(problem, pp, qq)
        dCs = der.dC(pp, qq)
        ip = int(np.ravel_multi_index(pp, M))
        iq = int(np.ravel_multi_index(qq, M))
        z = [np.zeros(d, complex), np.zeros(d, complex), np.zeros((d, d), complex)]
        z[0][ip] = 1.0
        z[1][iq] = 1.0
        # forward with checkpoints
        ckpt = {}
        for n in range(steps):
            if n % checkpoint_every == 0:
                ckpt[n] = [a.copy() for a in z]
            tau = n * dt
            O1, O2, O4 = ops(tau, 0.0), ops(tau, 0.5), ops(tau, 1.0)
            k1 = f(z, O1, C)
            k2 = f([a + 0.5 * dt * b for a, b in zip(z, k1)], O2, C)
            k3 = f([a + 0.5 * dt * b for a, b in zip(z, k2)], O2, C)
            k4 = f([a + dt * b for a, b in zip(z, k3)], O4, C)
            z = [a + (dt / 6.0) * (b1 + 2 * b2 + 2 * b3 + b4) for a, b1, b2, b3, b4 in zip(z, k1, k2, k3, k4)]
        G = np.outer(z[0], z[1]) + z[2]
        loss += (w * np.sum(lamG * G)).real
        # cotangent of the final state
        lam = [w * (lamG @ z[1]), w * (lamG.T @ z[0]), w * proj(lamG)]
        starts = sorted(ckpt)
        for s0 in reversed(starts):
            s1 = min(s0 + checkpoint_every, steps)
            # recompute the segment, keeping stage inputs
            zz = [a.copy() for a in ckpt[s0]]
            rec = []
            for n in range(s0, s1):
                tau = n * dt
                O1, O2, O4 = ops(tau, 0.0), ops(tau, 0.5), ops(tau, 1.0)
                u1 = zz
                k1 = f(u1, O1, C)
                u2 = [a + 0.5 * dt * b for a, b in zip(zz, k1)]
                k2 = f(u2, O2, C)
                u3 = [a + 0.5 * dt * b for a, b in zip(zz, k2)]
                k3 = f(u3, O2, C)
                u4 = [a + dt * b for a, b in zip(zz, k3)]
                k4 = f(u4, O4, C)
                rec.append((u1, u2, u3, u4, O1, O2, O4))
                zz = [a + (dt / 6.0) * (b1 + 2 * b2 + 2 * b3 + b4) for a, b1, b2, b3, b4 in zip(zz, k1, k2, k3, k4)]
            for n in reversed(range(s0, s1)):
                u1, u2, u3, u4, O1, O2, O4 = rec[n - s0]
                tau = n * dt
                b4 = [(dt / 6.0) * a for a in lam]
                q4 = JT(b4, u4, O4, C)
                param_dot(b4, u4, tau, 1.0, dCs)
                b3 = [(dt / 3.0) * a + dt * q for a, q in zip(lam, q4)]
                q3 = JT(b3, u3, O2, C)
                param_dot(b3, u3, tau, 0.5, dCs)
                b2 = [(dt / 3.0) * a + 0.5 * dt * q for a, q in zip(lam, q3)]
                q2 = JT(b2, u2, O2, C)
                param_dot(b2, u2, tau, 0.5, dCs)
                b1 = [(dt / 6.0) * a + 0.5 * dt * q for a, q in zip(lam, q2)]
                q1 = JT(b1, u1, O1, C)
                param_dot(b1, u1, tau, 0.0, dCs)
                lam = [a + x1 + x2 + x3 + x4 for a, x1, x2, x3, x4 in zip(lam, q1, q2, q3, q4)]
    return loss, grad_theta, grad_pwc


def loss_only(problem: Problem, M: Optional[Sequence[int]] = None, r_layout: str = "full") -> float:
    """l = Re Tr(rho0 A(T)) from oracle.mapping (used by finite differences)."""
    from .mapping import rk4_mapped
    from .fock import operator_matrix
    run = rk4_mapped(problem, M, r_layout=r_layout)
    A = run.fock_matrix()
    Mx = run.model.M
    rho = operator_matrix(problem.rho0_items(), Mx)
    return float(np.trace(rho @ A).real)


# ---- O3 for O1: the discrete adjoint of the number-basis RK4 solve ---------------------
def _direct_transpose(model, B: np.ndarray, H: np.ndarray) -> np.ndarray:
    """F^T(B) for the generator F(A) = i[H, A] + sum_n kappa_n (L^dag A L - 1/2 {L^dag L, A})
    (+ the secular dissipators) of Eq. 3, transposed under the bilinear pairing
    <B, A> = sum_kl B_kl A_kl: every product X A Y becomes X^T B Y^T."""
    out = 1j * (H.T @ B - B @ H.T)
    for rate, L, Ld, LdL in model.jumps:
        out += rate * (Ld.T @ B @ L.T - 0.5 * (LdL.T @ B + B @ LdL.T))
    if model.secular:
        # the secular terms K^dag A K, K A K^dag, P A, A P with real K and symmetric P
        # transpose to K B K^dag, K^dag B K, P B, B P: the Schroedinger form of the same
        # dissipator applied to B (evaluated padded and restricted like the adjoint)
        out += model.secular_schrodinger(B)
    return out


def loss_and_grad_direct(problem: Problem, N: Optional[Sequence[int]] = None, checkpoint_every: int = 64):
    """Loss l = Re Tr(rho0 A(T)) of the number-basis solve (oracle.fock.rk4_adjoint, O1) and
    its gradient by the exact discrete adjoint of classical RK4 on Eq. 3: with stage inputs
    u_i and the cotangent lam' of A(tau + h),
        b4 = h/6 lam', q_i = F_i^T(b_i), b3 = h/3 lam' + h q4, b2 = h/3 lam' + h/2 q3,
        b1 = h/6 lam' + h/2 q2, lam = lam' + q1 + q2 + q3 + q4,
        dl/dtheta += Re <b_i, i (dH/dtheta u_i - u_i dH/dtheta)>.
    Parameters as in loss_and_grad (H-term parameters, Re / Im of every piecewise-constant
    segment); the number-basis method has no separation constant.  Forward states are
    checkpointed every checkpoint_every steps and each segment is recomputed once.
    Returns (loss, dl/dtheta, {channel: (n_seg, 2)})."""
    from . import fock
    model = fock.FockModel(problem, N)
    Nm = model.N
    p = problem
    dt = p.dt
    steps = p.n_steps
    pad = 2 * _max_degree(problem) + 2
    big = tuple(n + pad for n in Nm)
    # every H term that carries a parameter or a channel, as its restricted matrix
    terms = []
    for t in p.h_terms:
        if t.param < 0 and t.channel < 0:
            continue
        m = kron_restricted(fock.monomial_factors(t.u, t.v, big), Nm)
        terms.append((m, complex(t.coef), t.param, t.channel, t.conj))
    grad_theta = np.zeros(len(p.params))
    grad_pwc: Dict[int, np.ndarray] = {}
    for ci, ch in enumerate(p.channels):
        if ch.kind == "pwc":
            grad_pwc[ci] = np.zeros(((len(ch.params) - 2) // 2, 2))
    rho = fock.operator_matrix(p.rho0_items(), Nm)
    lam_T = rho.T.copy()  # d Re Tr(rho0 A) / dA_kl = rho0_lk

    def F(A, H):
        return model.adjoint_generator(A, H)

    def param_dot(b, u, tau_step, c):
        for m, coef, param, chn, conj in terms:
            act = np.sum(b * (1j * (m @ u - u @ m)))  # <b, i [M_t, u]>
            theta = p.params[param] if param >= 0 else 1.0
            e = 1.0 + 0j
            if chn >= 0:
                e = stage_value(p.channels[chn], tau_step, c, dt, p.T, p.reverse_time)
                e = np.conj(e) if conj else e
            if param >= 0:
                grad_theta[param] += (coef * e * act).real
            if chn >= 0 and p.channels[chn].kind == "pwc":
                chd = p.channels[chn]
                tt = (p.T - (tau_step + 0.5 * dt)) if p.reverse_time else tau_step + 0.5 * dt
                s = int(math.floor((tt - chd.params[0]) / chd.params[1]))
                if 0 <= s < grad_pwc[chn].shape[0]:
                    g = coef * theta * act
                    grad_pwc[chn][s, 0] += g.real
                    grad_pwc[chn][s, 1] += (g * (-1j if conj else 1j)).real

    A = fock.operator_matrix(p.measured, Nm)
    ckpt = {}
    for n in range(steps):
        if n % checkpoint_every == 0:
            ckpt[n] = A.copy()
        tau = n * dt
        H1, H2, H4 = model.hamiltonian(tau, 0.0, dt), model.hamiltonian(tau, 0.5, dt), model.hamiltonian(tau, 1.0, dt)
        k1 = F(A, H1)
        k2 = F(A + 0.5 * dt * k1, H2)
        k3 = F(A + 0.5 * dt * k2, H2)
        k4 = F(A + dt * k3, H4)
        A = A + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    loss = float(np.sum(lam_T * A).real)
    lam = lam_T
    for s0 in reversed(sorted(ckpt)):
        s1 = min(s0 + checkpoint_every, steps)
        Z = ckpt[s0].copy()
        rec = []
        for n in range(s0, s1):
            tau = n * dt
            H1, H2, H4 = model.hamiltonian(tau, 0.0, dt), model.hamiltonian(tau, 0.5, dt), model.hamiltonian(tau, 1.0, dt)
            u1 = Z
            k1 = F(u1, H1)
            u2 = Z + 0.5 * dt * k1
            k2 = F(u2, H2)
            u3 = Z + 0.5 * dt * k2
            k3 = F(u3, H2)
            u4 = Z + dt * k3
            k4 = F(u4, H4)
            rec.append((u1, u2, u3, u4, H1, H2, H4))
            Z = Z + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        for n in reversed(range(s0, s1)):
            u1, u2, u3, u4, H1, H2, H4 = rec[n - s0]
            tau = n * dt
            b4 = (dt / 6.0) * lam
            q4 = _direct_transpose(model, b4, H4)
            param_dot(b4, u4, tau, 1.0)
            b3 = (dt / 3.0) * lam + dt * q4
            q3 = _direct_transpose(model, b3, H2)
            param_dot(b3, u3, tau, 0.5)
            b2 = (dt / 3.0) * lam + 0.5 * dt * q3
            q2 = _direct_transpose(model, b2, H2)
            param_dot(b2, u2, tau, 0.5)
            b1 = (dt / 6.0) * lam + 0.5 * dt * q2
            q1 = _direct_transpose(model, b1, H1)
            param_dot(b1, u1, tau, 0.0)
            lam = lam + q1 + q2 + q3 + q4
    return loss, grad_theta, grad_pwc


def loss_only_direct(problem: Problem, N: Optional[Sequence[int]] = None) -> float:
    """l = Re Tr(rho0 A(T)) from oracle.fock.rk4_adjoint (used by finite differences)."""
    from . import fock
    A = fock.rk4_adjoint(problem, N)
    Nm = tuple(N if N is not None else problem.N)
    rho = fock.operator_matrix(problem.rho0_items(), Nm)
    return float(np.trace(rho @ A).real)
