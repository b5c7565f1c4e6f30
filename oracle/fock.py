"""O1 -- the adjoint master equation (Eq. 3) on dense truncated number-basis matrices.

What it computes (the paper's "conventional approach"):
    dA/dtau = i[H(t), A] + sum_n kappa_n ( L_n^dag A L_n - 1/2 {L_n^dag L_n, A} ),
with classical RK4 (the integrator the paper uses for both methods) and, for the
Heisenberg picture of a time-dependent Hamiltonian, t = T - tau (see ``channels``).

Truncation reading: the generator is compressed onto operators supported on the span of
the first N_j Fock states of every mode; every operator that enters (H, L_n, L_n^dag L_n)
enters through its exact matrix elements in that span.  The matrices are therefore built
at a padded size and restricted, so that e.g. L^dag L for L = a^dag is diag(1..N), the
same as its normal-ordered form a^dag a + 1.

Secular dissipator (the paper's proper dissipator, Eq. 203 / Eq. S9, per damped mode j with
rate kappa and transition occupations nbar_n): with K_n = |n><n+1|_j (identity on the other
modes) and P_n = |n><n|_j,
    Schroedinger:  kappa/2 sum_n (nbar_n + 1)(n + 1) [2 K_n rho K_n^dag - {P_{n+1}, rho}]
                 + kappa/2 sum_n nbar_n (n + 1) [2 K_n^dag rho K_n - {P_n, rho}],
    adjoint:       the same with K_n rho K_n^dag -> K_n^dag A K_n and K_n^dag rho K_n -> K_n A K_n^dag.
Both are evaluated on A (rho) zero-padded by one level per mode and then restricted, the
same compression reading as for H and the jump operators.

Parity status (all pinned in tests/test_oracle_fock.py):
  * generator + RK4:      pinned by the damped-oscillator closed forms <a>(t), <a^dag a>(t);
                          by the binomial closed form for |m><m| under Kerr + damping;
                          by exact duality with the forward Schroedinger density-matrix RK4
                          (an independent code path) for time-dependent drives;
                          by the dense Liouvillian exponential (scipy.linalg.expm);
                          by unitary evolution U^dag A U for closed systems.
  * schrodinger_rk4:      pinned by the same duality and by trace preservation.
  * secular dissipator:   pinned (tests/test_oracle_secular.py) by equality with the
                          conventional dissipator on diagonal operators at zero temperature;
                          by the closed form A_{k,k+1}(t) = sqrt(k+1) exp(-(i Delta +
                          kappa (2k+1)/2) t) for A(0) = a; by adjoint / Schroedinger duality at
                          finite temperature with a drive; by unitality; by stationarity of
                          the thermal state rho_{n+1,n+1}/rho_{n,n} = nbar_n/(1 + nbar_n).
"""

from __future__ import annotations

from functools import reduce
from typing import List, Optional, Sequence, Tuple

import numpy as np

from workloads.spec import Problem
from .channels import channel_value, stage_value

RK4_C = (0.0, 0.5, 0.5, 1.0)


def ladder(n: int) -> np.ndarray:
    """Annihilation operator a on Fock states 0..n-1: a|k> = sqrt(k)|k-1>."""
    a = np.zeros((n, n), dtype=np.complex128)
    for k in range(1, n):
        a[k - 1, k] = np.sqrt(k)
    return a


def monomial_factors(u: Sequence[int], v: Sequence[int], dims: Sequence[int]) -> List[np.ndarray]:
    """Per-mode factors (a_j^dag)^u_j a_j^v_j of the monomial at the sizes `dims`."""
    mats = []
    for uj, vj, n in zip(u, v, dims):
        a = ladder(n)
        ad = a.conj().T
        mats.append(np.linalg.matrix_power(ad, uj) @ np.linalg.matrix_power(a, vj))
    return mats


def monomial(u: Sequence[int], v: Sequence[int], dims: Sequence[int]) -> np.ndarray:
    """prod_j (a_j^dag)^u_j a_j^v_j on the tensor product (mode 0 outermost)."""
    return reduce(np.kron, monomial_factors(u, v, dims))


def kron_restricted(factors: Sequence[np.ndarray], small: Sequence[int]) -> np.ndarray:
    """restrict(kron(factors), big, small) built factor by factor: the kept states (n_j <
    small_j in every mode) form a product sub-grid, on which a Kronecker product is the
    Kronecker product of the restricted factors (same entries, no full-size matrix)."""
    return reduce(np.kron, [f[:s, :s] for f, s in zip(factors, small)])


def restriction_indices(big: Sequence[int], small: Sequence[int]) -> np.ndarray:
    """Flat indices (in the 'big' tensor product) of the basis states with n_j < small_j."""
    grids = np.meshgrid(*[np.arange(s) for s in small], indexing="ij")
    flat = np.zeros(grids[0].shape, dtype=np.int64)
    for g, b in zip(grids, big):
        flat = flat * b + g
    return flat.reshape(-1)


def restrict(m: np.ndarray, big: Sequence[int], small: Sequence[int]) -> np.ndarray:
    idx = restriction_indices(big, small)
    return m[np.ix_(idx, idx)]


def _max_degree(problem: Problem) -> int:
    d = 0
    for t in problem.h_terms:
        d = max(d, sum(t.u) + sum(t.v))
    for j in problem.jumps:
        for _, u, v in j.terms:
            d = max(d, sum(u) + sum(v))
    return d


class FockModel:
    """Dense matrices of H's terms and of the jump operators, restricted to N per mode."""

    def __init__(self, problem: Problem, N: Optional[Sequence[int]] = None):
        self.p = problem
        self.N = tuple(N if N is not None else problem.N)
        pad = 2 * _max_degree(problem) + 2
        big = tuple(n + pad for n in self.N)
        self.dim = int(np.prod(self.N))

        def r(m):
            return restrict(m, big, self.N)

        self.h_static = np.zeros((self.dim, self.dim), dtype=np.complex128)
        self.h_dyn: List[Tuple[np.ndarray, int, bool, complex]] = []
        for t in problem.h_terms:
            c = complex(t.coef)
            if t.param >= 0:
                c *= problem.params[t.param]
            m = kron_restricted(monomial_factors(t.u, t.v, big), self.N)
            if t.channel < 0:
                self.h_static += c * m
            else:
                self.h_dyn.append((m, t.channel, t.conj, c))
        self.jumps = []  # (rate, L, L^dag, (L^dag L))
        for j in problem.jumps:
            # L = sum_t c_t M_t and L^dag L = sum_{s,t} conj(c_s) c_t M_s^dag M_t, every product
            # formed per mode at the padded size, then restricted
            fac = [(c, monomial_factors(u, v, big)) for c, u, v in j.terms]
            L = sum(c * kron_restricted(f, self.N) for c, f in fac)
            LdL = sum(np.conj(cs) * ct * kron_restricted([a.conj().T @ b for a, b in zip(fs, ft)], self.N)
                      for cs, fs in fac for ct, ft in fac)
            self.jumps.append((j.rate, L, L.conj().T, LdL))
        # secular dissipators: K_n, P_n, P_{n+1} on a space padded by one level per mode
        # (enough: they change a mode's level by at most one), with their weights
        sbig = tuple(n + 1 for n in self.N)
        self.big = sbig
        self.secular = []  # (kappa, [(w_down, w_up, K_n, P_n, P_n+1)])
        for sd in getattr(problem, "secular", []):
            ops = []
            for n in range(sbig[sd.mode] - 1):
                e = [np.eye(b, dtype=np.complex128) for b in sbig]
                kn = np.zeros((sbig[sd.mode], sbig[sd.mode]), dtype=np.complex128)
                kn[n, n + 1] = 1.0
                pn = np.zeros_like(kn)
                pn[n, n] = 1.0
                pn1 = np.zeros_like(kn)
                pn1[n + 1, n + 1] = 1.0

                def on_mode(m, e=e, j=sd.mode):
                    f = list(e)
                    f[j] = m
                    return reduce(np.kron, f)
                nb = sd.nbar_at(n)
                ops.append(((nb + 1.0) * (n + 1), nb * (n + 1), on_mode(kn), on_mode(pn), on_mode(pn1)))
            self.secular.append((sd.kappa, ops))
        self._ri = restriction_indices(sbig, self.N) if self.secular else None

    def _pad(self, X: np.ndarray) -> np.ndarray:
        d = int(np.prod(self.big))
        out = np.zeros((d, d), dtype=np.complex128)
        out[np.ix_(self._ri, self._ri)] = X
        return out

    def secular_adjoint(self, A: np.ndarray) -> np.ndarray:
        """Adjoint of the secular dissipators applied to A (padded, then restricted)."""
        if not self.secular:
            return np.zeros_like(A)
        Ab = self._pad(A)
        out = np.zeros_like(Ab)
        for kappa, ops in self.secular:
            for wd, wu, K, P, P1 in ops:
                Kd = K.conj().T
                out += 0.5 * kappa * wd * (2.0 * (Kd @ Ab @ K) - (P1 @ Ab + Ab @ P1))
                out += 0.5 * kappa * wu * (2.0 * (K @ Ab @ Kd) - (P @ Ab + Ab @ P))
        return out[np.ix_(self._ri, self._ri)]

    def secular_schrodinger(self, rho: np.ndarray) -> np.ndarray:
        """The secular dissipators of Eq. S9 applied to rho (padded, then restricted)."""
        if not self.secular:
            return np.zeros_like(rho)
        rb = self._pad(rho)
        out = np.zeros_like(rb)
        for kappa, ops in self.secular:
            for wd, wu, K, P, P1 in ops:
                Kd = K.conj().T
                out += 0.5 * kappa * wd * (2.0 * (K @ rb @ Kd) - (P1 @ rb + rb @ P1))
                out += 0.5 * kappa * wu * (2.0 * (Kd @ rb @ K) - (P @ rb + rb @ P))
        return out[np.ix_(self._ri, self._ri)]

    def hamiltonian(self, tau_step: float, c: float, dt: float) -> np.ndarray:
        p = self.p
        H = self.h_static.copy()
        for m, ch, conj, coef in self.h_dyn:
            e = stage_value(p.channels[ch], tau_step, c, dt, p.T, p.reverse_time)
            H += coef * (np.conj(e) if conj else e) * m
        return H

    def adjoint_generator(self, A: np.ndarray, H: np.ndarray) -> np.ndarray:
        """Right-hand side of Eq. 3 for the truncated operator A."""
        out = 1j * (H @ A - A @ H)
        for rate, L, Ld, LdL in self.jumps:
            out += rate * (Ld @ A @ L - 0.5 * (LdL @ A + A @ LdL))
        if self.secular:
            out += self.secular_adjoint(A)
        return out

    def schrodinger_generator(self, rho: np.ndarray, H: np.ndarray) -> np.ndarray:
        """Forward Lindblad equation, the dual of Eq. 3."""
        out = -1j * (H @ rho - rho @ H)
        for rate, L, Ld, LdL in self.jumps:
            out += rate * (L @ rho @ Ld - 0.5 * (LdL @ rho + rho @ LdL))
        if self.secular:
            out += self.secular_schrodinger(rho)
        return out


def operator_matrix(elems, N: Sequence[int]) -> np.ndarray:
    """Dense matrix from {(k tuple, l tuple): value}; entries outside the truncation are dropped."""
    dim = int(np.prod(N))
    A = np.zeros((dim, dim), dtype=np.complex128)
    for (k, l), val in elems.items():
        if all(kk < n for kk, n in zip(k, N)) and all(ll < n for ll, n in zip(l, N)):
            A[np.ravel_multi_index(k, N), np.ravel_multi_index(l, N)] += val
    return A


def rk4_adjoint(problem: Problem, N: Optional[Sequence[int]] = None, n_steps: Optional[int] = None,
                A0: Optional[np.ndarray] = None, record_every: int = 0):
    """Integrate Eq. 3 from tau = 0 with classical RK4; returns A(tau_end) (and records)."""
    model = FockModel(problem, N)
    A = operator_matrix(problem.measured, model.N) if A0 is None else A0.astype(np.complex128).copy()
    dt = problem.dt
    steps = problem.n_steps if n_steps is None else n_steps
    rec = []
    for n in range(steps):
        tau = n * dt
        H1 = model.hamiltonian(tau, 0.0, dt)
        H2 = model.hamiltonian(tau, 0.5, dt)
        H4 = model.hamiltonian(tau, 1.0, dt)
        k1 = model.adjoint_generator(A, H1)
        k2 = model.adjoint_generator(A + 0.5 * dt * k1, H2)
        k3 = model.adjoint_generator(A + 0.5 * dt * k2, H2)
        k4 = model.adjoint_generator(A + dt * k3, H4)
        A = A + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        if record_every and (n + 1) % record_every == 0:
            rec.append(A.copy())
    return (A, rec) if record_every else A


def schrodinger_rk4(problem: Problem, rho0: np.ndarray, N: Optional[Sequence[int]] = None,
                    n_steps: Optional[int] = None) -> np.ndarray:
    """Forward density-matrix RK4 in physical time t = 0..T (stages at t + c dt; the
    pwc envelope at the step midpoint), used to pin the Heisenberg reading."""
    model = FockModel(problem, N)
    p = problem
    dt = p.dt
    steps = p.n_steps if n_steps is None else n_steps
    rho = rho0.astype(np.complex128).copy()

    def ham(t_step, c):
        H = model.h_static.copy()
        for m, ch, conj, coef in model.h_dyn:
            chan = p.channels[ch]
            tt = t_step + 0.5 * dt if chan.kind == "pwc" else t_step + c * dt
            e = channel_value(chan, tt)
            H += coef * (np.conj(e) if conj else e) * m
        return H

    for n in range(steps):
        t = n * dt
        H1, H2, H4 = ham(t, 0.0), ham(t, 0.5), ham(t, 1.0)
        k1 = model.schrodinger_generator(rho, H1)
        k2 = model.schrodinger_generator(rho + 0.5 * dt * k1, H2)
        k3 = model.schrodinger_generator(rho + 0.5 * dt * k2, H2)
        k4 = model.schrodinger_generator(rho + dt * k3, H4)
        rho = rho + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return rho


def adjoint_liouvillian(problem: Problem, H: np.ndarray, N: Optional[Sequence[int]] = None) -> np.ndarray:
    """Dense superoperator of Eq. 3 acting on vec(A) (row-major flattening)."""
    model = FockModel(problem, N)
    d = model.dim
    I = np.eye(d)
    # vec_row(X A Y) = (X kron Y^T) vec_row(A)
    Lsup = 1j * (np.kron(H, I) - np.kron(I, H.T))
    for rate, L, Ld, LdL in model.jumps:
        Lsup += rate * (np.kron(Ld, L.T) - 0.5 * (np.kron(LdL, I) + np.kron(I, LdL.T)))
    if model.secular:  # column by column: the secular dissipators applied to every E_{ij}
        for c in range(d * d):
            E = np.zeros((d, d), dtype=np.complex128)
            E.reshape(-1)[c] = 1.0
            Lsup[:, c] += model.secular_adjoint(E).reshape(-1)
    return Lsup


def expectation(A: np.ndarray, rho: np.ndarray) -> complex:
    return complex(np.trace(rho @ A))


def low_block(A: np.ndarray, N: Sequence[int], lo: int = 3) -> np.ndarray:
    """Number-basis block with every mode index < lo (the paper's epsilon_r block)."""
    idx = restriction_indices(N, tuple(min(lo, n) for n in N))
    return A[np.ix_(idx, idx)]


def eps_r(M: np.ndarray, M_ref: np.ndarray) -> float:
    """Relative element-wise L2 error (the paper's epsilon_r)."""
    return float(np.linalg.norm(M - M_ref) / np.linalg.norm(M_ref))
