"""Plain FP64 CPU oracle of the DQMC fermion-weight engine for the 2D Holstein model.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU-baseline
leg of bench.py import, call or execute this package.  It shares no code with the CUDA
path: it has its own lattice set-up, propagators, stabilisation, update formulas,
measurements and Philox generator, and takes its inputs from workloads.py.

Paper: Li, Dee, Khatami, Johnston, "Accelerating lattice quantum Monte Carlo
simulations using artificial neural networks: an application to the Holstein model"
(arXiv:1905.07440).  Sections "Model" (the Hamiltonian H0 + H_lat + H_e-ph) and
"Determinant quantum Monte Carlo" (Trotter slicing, the weight
W = exp(-dtau S_ph) det M_up det M_dn with M = I + B_L ... B_1, the action S_ph, local
and block moves accepted with p = W(X')/W(X)).

Readings taken where the paper is silent (each also listed in the design notes):
  * B_l = exp(-dtau K) exp(-dtau V_l), V_l = diag(g X_l - mu): the -mu n term of H0 is
    kept with the diagonal factor.  det M is the same as for the paper's operator order.
  * G_l = (I + B_l ... B_1 B_L ... B_{l+1})^-1, G_ij = <c_i c_j^dagger>; the local move
    at slice l is evaluated on G_{l-1}, after which G is wrapped to G_l.
  * exp(-dtau K) is exact (dense eigendecomposition of K), no checkerboard.
  * K_ij = -t for every nearest-neighbour displacement (so a 2-site ring gets -2t).
  * Imaginary time is periodic in the phonon action: X_{i,L+1} = X_{i,1}.
  * Stabilisation (the paper defers to its refs): UDV by column-pivoted QR every
    n_wrap products, G from the UDV factors with the Db/Ds split; log|det M| from the
    same factors.  Here every restabilisation rebuilds the full product from X.
  * Visit order: local moves slice by slice, l = 1..L, sites i = 0..N-1 in index order;
    then one block move per site, i = 0..N-1.  Proposal widths: U[-dx_local, dx_local)
    and U[-dx_global, dx_global).  Accept iff u < p (u on the 2^-53 grid).
  * Measurements use the fresh G at each restabilised slice and are averaged per sweep;
    phonon averages use X at the end of the sweep.

Parity pins: see tests/test_oracle_pins.py (free-fermion and uniform-field closed forms,
atomic limit, particle-hole symmetry, brute-force determinants and ratios, Fock-space
expectation values, detailed balance, the free-phonon <X^2>).
"""
import math

import numpy as np
import scipy.linalg

from .philox import proposal_uniforms, TAG_LOCAL, TAG_GLOBAL


# ----------------------------------------------------------------------------- lattice

def site_index(x, y, nx):
    """Site numbering i = x + nx * y."""
    return x + nx * y


def hopping_matrix(p):
    """K with K_ij = -t summed over the four nearest-neighbour displacements (Model)."""
    N = p.nx * p.ny
    K = np.zeros((N, N))
    for y in range(p.ny):
        for x in range(p.nx):
            i = site_index(x, y, p.nx)
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                j = site_index((x + dx) % p.nx, (y + dy) % p.ny, p.nx)
                K[i, j] -= p.t
    return K


def kinetic_propagators(p):
    """(exp(-dtau K), exp(+dtau K)) from the symmetric eigendecomposition of K."""
    w, V = np.linalg.eigh(hopping_matrix(p))
    e_minus = (V * np.exp(-p.dtau * w)) @ V.T
    e_plus = (V * np.exp(p.dtau * w)) @ V.T
    return e_minus, e_plus


def slice_diagonal(p, x_l):
    """Diagonal of exp(-dtau V_l), V_l = diag(g X_l - mu)."""
    return np.exp(-p.dtau * (p.g * np.asarray(x_l) - p.mu))


def slice_matrix(p, expK, x_l):
    """B_l = exp(-dtau K) exp(-dtau V_l)."""
    return expK * slice_diagonal(p, x_l)[None, :]


# ------------------------------------------------------------------ stabilised products

def udv_chain(mats, n_wrap):
    """UDV factors of the product mats[-1] @ ... @ mats[0].

    Every n_wrap factors the running product P = (B ... B) U diag(D) is refactored by
    column-pivoted QR: P Pi = Q R, D = |diag R|, T' = D^-1 R Pi^T, so that
    P = Q diag(D) T'; then U <- Q and T <- T' T.
    """
    N = mats[0].shape[0]
    U = np.eye(N)
    D = np.ones(N)
    T = np.eye(N)
    for start in range(0, len(mats), n_wrap):
        P = U * D[None, :]
        for B in mats[start:start + n_wrap]:
            P = B @ P
        Q, R, piv = scipy.linalg.qr(P, pivoting=True)
        d = np.abs(np.diag(R))
        Tp = np.empty_like(R)
        Tp[:, piv] = R / d[:, None]
        T = Tp @ T
        U = Q
        D = d
    return U, D, T


def green_logdet_from_udv(U, D, T):
    """G = (I + U D T)^-1 and log|det(I + U D T)|.

    I + U D T = U Db (Db^-1 U^T + Ds T) with Db = max(D, 1), Ds = min(D, 1), so
    G = (Db^-1 U^T + Ds T)^-1 Db^-1 U^T and log|det| = sum log Db + log|det(...)|.
    """
    Db = np.maximum(D, 1.0)
    Ds = np.minimum(D, 1.0)
    rhs = U.T / Db[:, None]
    A = rhs + Ds[:, None] * T
    G = np.linalg.solve(A, rhs)
    _, ld = np.linalg.slogdet(A)
    return G, float(np.sum(np.log(Db)) + ld)


def slice_order(L, l):
    """0-based slice indices in application order for G_l: slices l+1..L, then 1..l."""
    return list(range(l, L)) + list(range(0, l))


def green_at(p, expK, X, l, n_wrap=None):
    """(G_l, log|det M|) for fields X[L][N], G_l = (I + B_l..B_1 B_L..B_{l+1})^-1, with QR every
    n_wrap products (default p.n_wrap)."""
    L = X.shape[0]
    mats = [slice_matrix(p, expK, X[s]) for s in slice_order(L, l % L)]
    return green_logdet_from_udv(*udv_chain(mats, n_wrap or p.n_wrap))


def log_det_M(p, expK, X, n_wrap=None):
    """log|det(I + B_L ... B_1)|."""
    return green_at(p, expK, X, 0, n_wrap)[1]


# ------------------------------------------------------------------------ phonon action

def phonon_action(p, X):
    """dtau * S_ph with S_ph = M/(2 dtau^2) sum (X_{l+1} - X_l)^2 + M Omega^2/2 sum X^2."""
    X = np.asarray(X)
    kin = np.sum((np.roll(X, -1, axis=0) - X) ** 2)
    pot = np.sum(X ** 2)
    return p.mass / (2.0 * p.dtau) * kin + 0.5 * p.dtau * p.mass * p.omega ** 2 * pot


def log_weight(p, expK, X):
    """log W(X) = 2 log|det M| - dtau S_ph (both spins share M)."""
    return 2.0 * log_det_M(p, expK, X) - phonon_action(p, X)


def local_action_change(p, X, s, i, x_new):
    """Change of dtau*S_ph when X[s, i] becomes x_new (neighbours s+1, s-1 periodic)."""
    L = X.shape[0]
    xo = X[s, i]
    xp = X[(s + 1) % L, i]
    xm = X[(s - 1) % L, i]
    kin = (xp - x_new) ** 2 + (x_new - xm) ** 2 - (xp - xo) ** 2 - (xo - xm) ** 2
    pot = x_new ** 2 - xo ** 2
    return p.mass / (2.0 * p.dtau) * kin + 0.5 * p.dtau * p.mass * p.omega ** 2 * pot


def global_action_change(p, X, i, dx):
    """Change of dtau*S_ph when X[:, i] is shifted by dx (the kinetic term is unchanged)."""
    col = X[:, i]
    return 0.5 * p.dtau * p.mass * p.omega ** 2 * float(np.sum((col + dx) ** 2 - col ** 2))


def _exp(x):
    return math.exp(min(x, 709.0))


# ------------------------------------------------------------------------ measurements

def staggered_signs(p):
    s = np.empty(p.nx * p.ny)
    for y in range(p.ny):
        for x in range(p.nx):
            s[site_index(x, y, p.nx)] = -1.0 if (x + y) % 2 else 1.0
    return s


def measure_green(p, G):
    """Equal-time electronic observables from G (Wick's theorem, both spins alike).

    <n_i> = 2 (1 - G_ii);  <n_i,up n_i,dn> = (1 - G_ii)^2;
    <n_i n_j> = 4 (1 - G_ii)(1 - G_jj) + 2 delta_ij G_ii - 2 G_ij G_ji;
    S_CDW(pi, pi) = (1/N) sum_ij (-1)^(i+j) <n_i n_j>.
    """
    N = G.shape[0]
    m = 1.0 - np.diag(G)
    s = staggered_signs(p)
    conn = np.sum(np.outer(s, s) * G * G.T)
    scdw = (4.0 * (s @ m) ** 2 + 2.0 * np.sum(np.diag(G)) - 2.0 * conn) / N
    return dict(density=2.0 * float(np.mean(m)), double_occ=float(np.mean(m * m)),
                s_cdw=float(scdw))


def measure_fields(X):
    return dict(x_mean=float(np.mean(X)), x2=float(np.mean(X * X)))


OBSERVABLES = ("density", "double_occ", "s_cdw", "x_mean", "x2")


# ------------------------------------------------------------------------------ chain

class OracleChain:
    """One Markov chain of the plain DQMC sampler (local sweep, then block moves)."""

    def __init__(self, p, X, chain=0, sweep=0, record=False):
        self.p = p
        self.X = np.array(X, dtype=np.float64, copy=True)
        assert self.X.shape == (p.n_slices, p.n_sites)
        assert p.n_slices >= 2
        self.chain = int(chain)
        self.sweep_index = int(sweep)
        self.expK, self.expKinv = kinetic_propagators(p)
        self.n_wrap = p.n_wrap
        self.G, self.logdet = green_at(p, self.expK, self.X, 0)
        self.record = record
        self.moves = []
        self.wrap_exceeded = 0
        self.unstable = False

    # -- local moves with the fast (rank-1) update, then the wrap
    def local_sweep(self, measure=True):
        p, X = self.p, self.X
        L, N = X.shape
        G = self.G
        acc = 0
        max_err = 0.0
        meas = []
        ld = self.logdet
        for s in range(L):
            u1, u2 = proposal_uniforms(p.seed, self.chain, self.sweep_index,
                                       s * N + np.arange(N), TAG_LOCAL)
            for i in range(N):
                dx = p.dx_local * (2.0 * u1[i] - 1.0)
                x_new = X[s, i] + dx
                delta = math.exp(-p.dtau * p.g * dx) - 1.0
                R1 = 1.0 + delta * (1.0 - G[i, i])
                dS = local_action_change(p, X, s, i, x_new)
                prob = R1 * R1 * _exp(-dS)
                accepted = bool(u2[i] < prob)
                if self.record:
                    self.moves.append(dict(kind="local", s=s, i=i, dx=dx, log_ratio=2.0 * math.log(abs(R1)),
                                           dS=dS, accepted=accepted, X_before=None if not accepted else X.copy()))
                if accepted:
                    col = G[:, i].copy()
                    col[i] -= 1.0
                    row = G[i, :].copy()
                    G = G + (delta / R1) * np.outer(col, row)
                    X[s, i] = x_new
                    acc += 1
            d = slice_diagonal(p, X[s])
            G = self.expK @ ((d[:, None] * G) / d[None, :]) @ self.expKinv
            l = s + 1
            if l % self.n_wrap == 0 or l == L:
                Gf, ld = green_at(p, self.expK, X, l, self.n_wrap)
                max_err = max(max_err, float(np.max(np.abs(G - Gf))))
                G = Gf
                if measure:
                    meas.append(measure_green(p, Gf))
        self.G = G
        self.logdet = ld
        out = dict(local_accepted=acc, max_wrap_error=max_err)
        if measure:
            for k in meas[0]:
                out[k] = float(np.mean([m[k] for m in meas]))
        return out

    # -- block moves: one per site, each with the full stabilised determinant
    def global_sweep(self, sites=0):
        """sites > 0 (and < N): only a run of `sites` consecutive sites (index order, periodic)
        from j0 = floor(u N), u the first uniform of event N of this sweep's block-move stream."""
        p, X = self.p, self.X
        L, N = X.shape
        u1, u2 = proposal_uniforms(p.seed, self.chain, self.sweep_index, np.arange(N + 1), TAG_GLOBAL)
        order = list(range(N))
        if 0 < sites < N:
            j0 = min(int(float(u1[N]) * N), N - 1)
            order = [(j0 + k) % N for k in range(sites)]
        ld = self.logdet
        acc = 0
        for i in order:
            dx = p.dx_global * (2.0 * u1[i] - 1.0)
            dS = global_action_change(p, X, i, dx)
            Xn = X.copy()
            Xn[:, i] += dx
            ldn = log_det_M(p, self.expK, Xn, self.n_wrap)
            prob = _exp(2.0 * (ldn - ld) - dS)
            accepted = bool(u2[i] < prob)
            if self.record:
                self.moves.append(dict(kind="global", s=None, i=i, dx=dx, log_ratio=2.0 * (ldn - ld),
                                       dS=dS, accepted=accepted, X_before=None if not accepted else X.copy()))
            if accepted:
                X = Xn
                ld = ldn
                acc += 1
        self.X = X
        self.G, self.logdet = green_at(p, self.expK, X, 0, self.n_wrap)
        return dict(global_accepted=acc)

    def sweep(self, do_local=True, do_global=True, measure=True, block_sites=0):
        out = {}
        if do_local:
            out.update(self.local_sweep(measure=measure))
        if do_global:
            out.update(self.global_sweep(sites=block_sites))
        if measure:
            out.update(measure_fields(self.X))
        self.sweep_index += 1
        if do_local and getattr(self.p, "wrap_tol", 0.0) > 0.0:
            self._backoff(out["max_wrap_error"])
        return out

    def _backoff(self, err):
        """Stabilisation back-off (reading of the design notes; the paper defers stabilisation to
        its references): a sweep whose largest |G_wrapped - G_fresh| exceeds wrap_tol halves the
        restabilisation interval for the following sweeps, down to n_wrap_min; at that floor the
        chain is reported unstable."""
        if err <= self.p.wrap_tol:
            return
        self.wrap_exceeded += 1
        floor = self.p.n_wrap_min if self.p.n_wrap_min > 0 else 1
        if self.n_wrap <= floor:
            self.unstable = True
        else:
            self.n_wrap = max(floor, self.n_wrap // 2)

    def log_weight(self):
        return 2.0 * self.logdet - phonon_action(self.p, self.X)


def run_chains(p, X0, n_sweeps, first_chain=0, sweep0=0, do_local=True, do_global=True):
    """Run independent chains; returns final X, G, logdet and per-sweep records."""
    C = X0.shape[0]
    Xs, Gs, lds, recs = [], [], [], []
    for c in range(C):
        ch = OracleChain(p, X0[c], chain=first_chain + c, sweep=sweep0)
        r = [ch.sweep(do_local=do_local, do_global=do_global) for _ in range(n_sweeps)]
        Xs.append(ch.X)
        Gs.append(ch.G)
        lds.append(ch.logdet)
        recs.append(r)
    return np.array(Xs), np.array(Gs), np.array(lds), recs
